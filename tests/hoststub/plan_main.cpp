// Builds plans of 1, 2, 3 and 8 streams, retiles and "executes" them (test only).
#include "dpd.h"
#include <cstdio>
#include <vector>
#include <complex>
int main() {
  for (int count : {1, 2, 3, 8}) {
    std::vector<std::vector<std::complex<float>>> xs(count), ys(count), hs(count);
    std::vector<dpd_stream_desc> d(count);
    for (int i = 0; i < count; ++i) {
      int n = 100000 / (i + 1); xs[i].resize(n + 2); ys[i].resize(n + 2); hs[i].resize(97);
      d[i] = {xs[i].data(), ys[i].data(), n, 5, 5, 3, hs[i].data()};
    }
    dpd_plan p = nullptr;
    int rc = dpd_plan_batched(d.data(), count, DPD_HOST, &p);
    printf("count %d rc %d\n", count, rc);
    if (p) {
      rc = dpd_plan_set_launch(p, 4, 8, 4, 0, 0); printf(" set_launch %d\n", rc); rc = dpd_exec_batched(p, nullptr); printf(" exec %d\n", rc);
      rc = dpd_plan_set_launch(p, 8, 12, 3, 0, 4); printf(" set_launch grouped %d\n", rc); rc = dpd_exec_batched(p, nullptr); printf(" exec %d\n", rc);
      rc = dpd_plan_set_launch(p, 8, 12, 3, 0, 5); printf(" set_launch bad group %d\n", rc);
      dpd_plan_destroy(p);
    }
  }
}
