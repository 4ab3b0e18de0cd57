// Level-symmetric (LQn) discrete-ordinate sets on the host (Sec. 2, after eq. 2: positive
// weights summing to 4 pi; the paper's results use level-symmetric S2 / S4 sets).
//
// Construction: direction cosines mu_i^2 = mu_1^2 + (i - 1) 2 (1 - 3 mu_1^2) / (N - 2),
// i = 1..N/2; the directions of one octant are the level-index triples (i, j, k) with
// i + j + k = N/2 + 2, each carrying the weight of its permutation class; the class weights
// are normalised so that an octant sums to 1.  mu_1 and the class weights are the published
// 7-digit LQn table values.  Compiled with -ffp-contract=off, every value follows the stated
// operation order (the octant sum is taken left to right in point order).
#include <cmath>
#include <cstring>
#include <vector>
#include "common.h"

namespace {

struct LQn {
  int N;
  double mu1;
  int n_classes;
  int cls[5][3];        // sorted 1-based level-index triples
  double wt[5];         // point weight of each class within an octant (before normalisation)
};

const LQn kSets[] = {
    {2, 0.5773502691896257, 1, {{1, 1, 1}}, {1.0}},
    {4, 0.3500212, 1, {{1, 1, 2}}, {1.0 / 3.0}},
    {6, 0.2666355, 2, {{1, 1, 3}, {1, 2, 2}}, {0.1761263, 0.1572071}},
    {8, 0.2182179, 3, {{1, 1, 4}, {1, 2, 3}, {2, 2, 2}}, {0.1209877, 0.0907407, 0.0925926}},
    {12, 0.1672126, 5, {{1, 1, 6}, {1, 2, 5}, {1, 3, 4}, {2, 2, 4}, {2, 3, 3}},
     {0.0707626, 0.0558811, 0.0373377, 0.0502819, 0.0258513}},
};

double class_weight(const LQn& s, int a, int b, int c) {
  int t[3] = {a, b, c};
  // sort the triple ascending
  for (int x = 0; x < 3; ++x)
    for (int y = x + 1; y < 3; ++y)
      if (t[y] < t[x]) {
        const int tmp = t[x];
        t[x] = t[y];
        t[y] = tmp;
      }
  for (int k = 0; k < s.n_classes; ++k)
    if (s.cls[k][0] == t[0] && s.cls[k][1] == t[1] && s.cls[k][2] == t[2]) return s.wt[k];
  return -1.0;
}

}  // namespace

extern "C" sn_status sn_quadrature_level_symmetric(int N, int dim, int* n_dir, double* omega, double* w) {
  if (!n_dir || (dim != 2 && dim != 3)) return SN_EINVAL;
  const LQn* s = nullptr;
  for (const LQn& c : kSets)
    if (c.N == N) s = &c;
  if (!s) return SN_EINVAL;
  const int n = N / 2;
  std::vector<double> mu(n);
  if (N == 2) {
    mu[0] = s->mu1;
  } else {
    for (int i = 0; i < n; ++i) {
      const double m2 = s->mu1 * s->mu1 + i * 2.0 * (1.0 - 3.0 * s->mu1 * s->mu1) / (N - 2);
      mu[i] = std::sqrt(m2);
    }
  }
  // octant points: level-index triples with i + j + k = n + 2, i fastest, then j, then k
  std::vector<int> pi, pj, pk;
  std::vector<double> pw;
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i)
        if (i + j + k == n + 2) {
          pi.push_back(i);
          pj.push_back(j);
          pk.push_back(k);
          pw.push_back(class_weight(*s, i, j, k));
        }
  double tot = 0.0;
  for (double x : pw) tot += x;
  for (double& x : pw) x = x / tot;
  const int npt = (int)pw.size();
  const int noct = dim == 3 ? 8 : 4;
  const double scale = dim == 3 ? M_PI / 2.0 : M_PI;
  *n_dir = npt * noct;
  if (!omega && !w) return SN_OK;
  if (!omega || !w) return SN_EINVAL;
  // octants in sign order (+,+,+), (-,+,+), (+,-,+), (-,-,+), then z < 0 in 3D
  for (int o = 0; o < noct; ++o) {
    const double sx = (o & 1) ? -1.0 : 1.0, sy = (o & 2) ? -1.0 : 1.0, sz = (o & 4) ? -1.0 : 1.0;
    for (int q = 0; q < npt; ++q) {
      const int d = o * npt + q;
      omega[3 * d + 0] = mu[pi[q] - 1] * sx;
      omega[3 * d + 1] = mu[pj[q] - 1] * sy;
      omega[3 * d + 2] = mu[pk[q] - 1] * sz;
      w[d] = pw[q] * scale;
    }
  }
  return SN_OK;
}
