// Host check of the small dense routines of libmhde, driven from
// tests/test_host_small_dense_cpu.py through stdin/stdout:
//   "L r J m S0 h_0 ... h_{m-1}"  -> block least squares (BlockLS): after each
//                                    block column its ok flag and the J residual
//                                    norms, then the solution (m r x J)
//   "Q r thresh g_00 ... g_rr"    -> Cholesky QR factors of a Gram matrix: the
//                                    accepted flag, then T (r x r) and S (r x r)
#include <cstdio>
#include <vector>

#include "../../paper_2108_05110_gb300/csrc/mhde_internal.h"

int main() {
  char mode[8];
  int n;
  while (std::scanf("%7s %d", mode, &n) == 2) {
    if (mode[0] == 'L') {
      const int r = n;
      int J = 0, m = 0;
      if (std::scanf("%d %d", &J, &m) != 2) return 1;
      std::vector<double> S0((size_t)r * J);
      for (auto& v : S0) std::scanf("%lf", &v);
      mhde::BlockLS ls;
      ls.init(r, J, m, S0.data());
      for (int k = 0; k < m; ++k) {
        std::vector<double> h((size_t)(k + 2) * r * r);
        for (auto& v : h) std::scanf("%lf", &v);
        const bool ok = ls.add(h.data());
        std::printf("%d", ok ? 1 : 0);
        for (int j = 0; j < J; ++j) std::printf(" %.17g", ls.resid(j));
        std::printf("\n");
      }
      std::vector<double> Y;
      ls.solve(Y);
      for (double v : Y) std::printf("%.17g\n", v);
    } else if (mode[0] == 'Q') {
      const int r = n;
      double thresh = 0.0;
      if (std::scanf("%lf", &thresh) != 1) return 1;
      std::vector<double> G((size_t)r * r), T, S;
      for (auto& v : G) std::scanf("%lf", &v);
      const bool ok = mhde::cholqr_factors(r, G, thresh, T, S);
      std::printf("%d\n", ok ? 1 : 0);
      if (ok) {
        for (double v : T) std::printf("%.17g\n", v);
        for (double v : S) std::printf("%.17g\n", v);
      }
    } else {
      return 1;
    }
  }
  return 0;
}
