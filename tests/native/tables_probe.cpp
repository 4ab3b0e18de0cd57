// Prints the host tables of one element family (tables.cpp) as text for the CPU test
// test_host_tables.py, which compares them with the oracle's.  Usage: tables_probe FAMILY P R
// with FAMILY one of tensor2, tensor3, tri, tet.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "../../paper_1810_11080_gb300/csrc/common.h"

static void put(const char* name, const std::vector<double>& v) {
  std::printf("%s %zu", name, v.size());
  for (double x : v) std::printf(" %.17g", x);
  std::printf("\n");
}

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  const char* fam = argv[1];
  const int p = std::atoi(argv[2]), r = std::atoi(argv[3]);
  sn::Tables T;
  if (!std::strcmp(fam, "tensor2")) sn::build_tables(T, 2, p, r);
  else if (!std::strcmp(fam, "tensor3")) sn::build_tables(T, 3, p, r);
  else if (!std::strcmp(fam, "tri")) sn::build_tables_tri(T, p, r);
  else if (!std::strcmp(fam, "tet")) sn::build_tables_tet(T, p);
  else return 2;
  std::printf("dims %d %d %d %d %d %d %d\n", T.nv, T.nf, T.N, T.Nf, T.Nv, T.Q, T.dim);
  put("glv_t", T.glv_t);
  put("glv_w", T.glv_w);
  put("glf_t", T.glf_t);
  put("glf_w", T.glf_w);
  put("wq", T.wq);
  put("B", T.B);
  put("dB", T.dB);
  put("V", T.V);
  put("dV", T.dV);
  return 0;
}
