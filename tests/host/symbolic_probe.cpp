// Test probe (not part of the library): runs the host set-up of a mesh
// (edges, PEC removal, nested dissection, fronts) without a GPU and writes
// what the symbolic checks need, in native binary:
//   int64 N, int64 nt, int32 tdof[nt*6], int64 nfront,
//   per front: int32 k, n, c0, parent, height, ld, int64 lofs, uofs, then
//   n - k int32 update rows and (non-root fronts) n - k int32 positions of
//   those rows in the parent front (the extend-add relative map),
//   then int64 nnz_l (factor entries per pole), ltotal, utotal, the CSR of A in
//   the elimination order (int64 rp[N+1], int64 nnz, int32 ci[nnz]) and the
//   map of A's lower-triangle entries to factor positions (int64 no,
//   int64 orig_nz[no], int64 orig_dst[no]), then the levels (int64 nl; per
//   level int64 nfront and int32 fronts[nfront], int64 ea_beg[4], ea_end[4]) and the
//   extend-add tasks (int64 nea, int32 ea_child[nea], int32 ea_col[nea]).
// Input (argv[1], native binary): int64 nv, int64 nt, int32 leaf_max, int32 amalg_max,
// double xyz[nv*3], int32 tets[nt*4], double sigma[nt], uint8 is_param[nt].
#include <cstdio>
#include <vector>
#include "tem_internal.h"

int main(int argc, char **argv) {
  if (argc != 3) return 2;
  FILE *f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t nv = 0, nt = 0;
  int32_t leaf = 0, amalg = 0;
  bool ok = std::fread(&nv, 8, 1, f) == 1 && std::fread(&nt, 8, 1, f) == 1 && std::fread(&leaf, 4, 1, f) == 1 &&
            std::fread(&amalg, 4, 1, f) == 1;
  std::vector<double> xyz(3 * nv > 0 ? 3 * nv : 0), sig(nt > 0 ? nt : 0);
  std::vector<int32_t> tets(4 * nt > 0 ? 4 * nt : 0);
  std::vector<uint8_t> ip(nt > 0 ? nt : 0);
  ok = ok && std::fread(xyz.data(), 8, xyz.size(), f) == xyz.size() &&
       std::fread(tets.data(), 4, tets.size(), f) == tets.size() && std::fread(sig.data(), 8, sig.size(), f) == sig.size() &&
       std::fread(ip.data(), 1, ip.size(), f) == ip.size();
  std::fclose(f);
  if (!ok) return 2;
  tem::Mesh m;
  tem::Symbolic s;
  const std::string e = tem::build_mesh(m, nv, xyz.data(), nt, tets.data(), sig.data(), ip.data(), tem::SymOpts{leaf, amalg}, s);
  if (!e.empty()) {
    std::fprintf(stderr, "%s\n", e.c_str());
    return 1;
  }
  FILE *o = std::fopen(argv[2], "wb");
  if (!o) return 2;
  const int64_t nf = (int64_t)s.fronts.size();
  std::fwrite(&m.N, 8, 1, o);
  std::fwrite(&m.nt, 8, 1, o);
  std::fwrite(m.tdof.data(), 4, m.tdof.size(), o);
  std::fwrite(&nf, 8, 1, o);
  for (const tem::Front &F : s.fronts) {
    const int32_t h[6] = {F.k, F.n, F.c0, F.parent, F.height, F.ld};
    const int64_t offs[2] = {F.lofs, F.uofs};
    std::fwrite(h, 4, 6, o);
    std::fwrite(offs, 8, 2, o);
    std::fwrite(s.rows.data() + F.rows_off, 4, F.n - F.k, o);
    if (F.parent >= 0) std::fwrite(s.rel.data() + F.rel_off, 4, F.n - F.k, o);
  }
  std::fwrite(&s.nnz_l, 8, 1, o);
  std::fwrite(&s.ltotal, 8, 1, o);
  std::fwrite(&s.utotal, 8, 1, o);
  const int64_t nnz = (int64_t)m.ci.size(), no = (int64_t)s.orig_nz.size();
  std::fwrite(m.rp.data(), 8, m.rp.size(), o);
  std::fwrite(&nnz, 8, 1, o);
  std::fwrite(m.ci.data(), 4, m.ci.size(), o);
  std::fwrite(&no, 8, 1, o);
  std::fwrite(s.orig_nz.data(), 8, s.orig_nz.size(), o);
  std::fwrite(s.orig_dst.data(), 8, s.orig_dst.size(), o);
  const int64_t nl = (int64_t)s.levels.size(), nea = (int64_t)s.ea_child.size();
  std::fwrite(&nl, 8, 1, o);
  for (const tem::Level &L : s.levels) {
    const int64_t nfl = (int64_t)L.fronts.size();
    std::fwrite(&nfl, 8, 1, o);
    std::fwrite(L.fronts.data(), 4, L.fronts.size(), o);
    std::fwrite(L.ea_beg, 8, tem::kMaxChild, o);
    std::fwrite(L.ea_end, 8, tem::kMaxChild, o);
  }
  std::fwrite(&nea, 8, 1, o);
  std::fwrite(s.ea_child.data(), 4, s.ea_child.size(), o);
  std::fwrite(s.ea_col.data(), 4, s.ea_col.size(), o);
  std::fclose(o);
  return 0;
}
