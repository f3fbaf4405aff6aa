// Host program for tests/test_sort_curves.py: prints, for each curve (0 =
// Morton, 1 = Hilbert) and each b in 1..5, the number of keys that are not
// a permutation of [0, 8^b) and the number of consecutive key pairs whose
// buckets are not face neighbours.  Uses the same curve_key3 as the kernels.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "k_device.cuh"

int main() {
  for (int hilbert = 0; hilbert < 2; ++hilbert) {
    for (int b = 1; b <= 5; ++b) {
      const unsigned n = 1u << b, N = n * n * n;
      std::vector<int> where(N, -1);
      long bad_perm = 0, jumps = 0;
      for (unsigned z = 0; z < n; ++z)
        for (unsigned y = 0; y < n; ++y)
          for (unsigned x = 0; x < n; ++x) {
            const unsigned k = crash::curve_key3(x, y, z, b, hilbert != 0);
            if (k >= N || where[k] >= 0) { ++bad_perm; continue; }
            where[k] = (int)(x | (y << 10) | (z << 20));
          }
      for (unsigned k = 1; k < N; ++k) {
        if (where[k] < 0 || where[k - 1] < 0) continue;
        const int a = where[k - 1], c = where[k];
        const int d = std::abs((a & 1023) - (c & 1023)) + std::abs(((a >> 10) & 1023) - ((c >> 10) & 1023)) +
                      std::abs((a >> 20) - (c >> 20));
        if (d != 1) ++jumps;
      }
      std::printf("%d %d %ld %ld\n", hilbert, b, bad_perm, jumps);
    }
  }
  return 0;
}
