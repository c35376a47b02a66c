// Exact 1-D Galerkin masks of the re-discretised coarse operators (Section 3.3, Appendix A).
//
// The level-l stencils are Lap_l = (L_l (x) M_l + M_l (x) L_l) / h^2 and K_l = M_l (x) M_l
// with 1-D masks obtained by Galerkin coarsening with the deflation weights
// p = [1, 4, 6, 4, 1] / 8 at stride 2:  S_{l+1}[d] = sum_{a,e} p_a S_l[e] p_{a+e-2d},
// from M_1 = [1], L_1 = [-1, 2, -1].  The masks are carried as integer numerators over the
// common denominator 64^(l-1) (exact), then rounded once to double.
#include <cstdint>
#include <vector>

#include "hz_internal.h"

namespace hz {

namespace {
typedef __int128 i128;

// One Galerkin step on integer numerators (denominator grows by 64).
std::vector<i128> coarsen(const std::vector<i128>& s) {
  static const int P[5] = {1, 4, 6, 4, 1};
  const int rs = (int)s.size() / 2;
  const int rc = rs / 2 + 2;  // support of the coarse stencil
  std::vector<i128> out(2 * rc + 1, 0);
  for (int d = -rc; d <= rc; ++d) {
    i128 acc = 0;
    for (int a = -2; a <= 2; ++a)
      for (int e = -rs; e <= rs; ++e) {
        int m = a + e - 2 * d;
        if (m >= -2 && m <= 2) acc += (i128)P[a + 2] * s[e + rs] * P[m + 2];
      }
    out[d + rc] = acc;
  }
  // trim zero tails symmetrically
  int r = rc;
  while (r > 0 && out[0] == 0 && out[out.size() - 1] == 0) {
    out.erase(out.begin());
    out.pop_back();
    --r;
  }
  return out;
}
}  // namespace

void galerkin_masks(int level, int* R, double m[7], double l[7]) {
  std::vector<i128> mm = {1}, ll = {-1, 2, -1};
  double den = 1.0;
  for (int i = 1; i < level; ++i) {
    mm = coarsen(mm);
    ll = coarsen(ll);
    den *= 64.0;
  }
  int rm = (int)mm.size() / 2, rl = (int)ll.size() / 2;
  int r = rm > rl ? rm : rl;
  *R = r;
  for (int i = 0; i < 7; ++i) m[i] = l[i] = 0.0;
  for (int d = -r; d <= r; ++d) {
    i128 a = (d >= -rm && d <= rm) ? mm[d + rm] : 0;
    i128 b = (d >= -rl && d <= rl) ? ll[d + rl] : 0;
    m[d + r] = (double)a / den;
    l[d + r] = (double)b / den;
  }
}

}  // namespace hz
