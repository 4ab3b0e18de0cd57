// Prints the tetrahedron node maps of the sweep kernels (devmath.cuh, the TetEl policy and its
// packed tables in inverse_body.cuh), evaluated on the host, for test_host_tables.py.
#include <cstdio>
#include "../../paper_1810_11080_gb300/csrc/common.h"
#include "../../paper_1810_11080_gb300/csrc/sweep_kernels.cuh"

template <int P>
static void dump() {
  constexpr auto tw = sn::tet_trace_words<P>();
  for (int f = 0; f < 4; ++f) {
    std::printf("face %d %d", P, f);
    for (int j = 0; j < sn::TetEl<P>::NF; ++j) std::printf(" %d", sn::TetEl<P>::vol_node(f, j));
    std::printf("\nfaceword %d %d %llu\n", P, f, (unsigned long long)sn::TetEl<P>::face_node_word(f));
  }
  for (int k = 0; k < 24; ++k) std::printf("trace %d %d %u\n", P, k, tw.w[k]);
}

int main() {
  dump<1>();
  dump<2>();
  return 0;
}
