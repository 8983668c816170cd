// Host harness for the fixed-point accumulator of the packed S-apply (cpm_fixed.cuh): reads a
// split point k, a count n and n float32 bit patterns (hex) from stdin, adds values [0, k) into one
// accumulator and [k, n) into another, merges them, and prints the float64 value and the 128-bit
// state (hex, high then low word).
#include <cstdio>
#include <cstring>

#include "../paper_2201_12963_gb300/csrc/cpm_fixed.cuh"

int main() {
  int k = 0, n = 0;
  if (std::scanf("%d %d", &k, &n) != 2) return 1;
  cpm::Fx128 a, b;
  for (int i = 0; i < n; ++i) {
    unsigned int u;
    if (std::scanf("%x", &u) != 1) return 1;
    float x;
    std::memcpy(&x, &u, sizeof(x));
    (i < k ? a : b).add(x);
  }
  a.add(b);
  std::printf("%.17g %016llx %016llx\n", a.value(), a.hi, a.lo);
  return 0;
}
