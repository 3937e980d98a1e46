// Host check of the contraction's weighted tile split (ctd_contract_tc.cuh): CTA c owns the
// tiles [tile_lo(c), tile_lo(c + 1)); the first 16 CTAs weigh 1, the others 8.  Brute force
// over many tile counts T and grid sizes G:
//   * the ranges partition [0, T) in order;
//   * tile_owner(t) is the CTA whose range holds t, for every t;
//   * each CTA's share is within one tile of T w(c) / sum w;
//   * tile_div equals 64-bit division on both sides of its 32-bit fast path.
// Prints one line per failure and exits 1 if there is any.
#include "ctd_contract_tc.cuh"

#include <cstdio>
#include <cstdlib>

static int failures = 0;

static void fail(const char* what, long long T, int G, long long a, long long b) {
  if (failures < 20) std::printf("FAIL %s T=%lld G=%d %lld %lld\n", what, T, G, a, b);
  ++failures;
}

static void check(long long T, int G) {
  using namespace ctd;
  if (tile_lo(T, G, 0) != 0) fail("lo(0)", T, G, tile_lo(T, G, 0), 0);
  if (tile_lo(T, G, G) != T) fail("lo(G)", T, G, tile_lo(T, G, G), T);
  const int L = G < kLightCtas ? G : kLightCtas;
  const double tot = static_cast<double>(L) + static_cast<double>(kHeavyWeight) * (G - L);
  for (int c = 0; c < G; ++c) {
    const long long lo = tile_lo(T, G, c), hi = tile_lo(T, G, c + 1);
    if (hi < lo) fail("order", T, G, c, hi - lo);
    const double share = static_cast<double>(T) * (c < L ? 1.0 : kHeavyWeight) / tot;
    if (hi - lo > share + 1.0 || hi - lo < share - 1.0) fail("share", T, G, c, hi - lo);
    for (long long t = lo; t < hi; ++t)
      if (tile_owner(T, G, t) != c) fail("owner", T, G, t, tile_owner(T, G, t));
  }
}

int main() {
  const int grids[] = {1, 2, 3, 5, 15, 16, 17, 18, 31, 64, 100, 151, 152, 304};
  const long long tiles[] = {1, 2, 3, 7, 16, 17, 100, 151, 152, 153, 1000, 1024, 4096, 8191,
                             65536, 262144, 4000000, 9000000};
  for (int G : grids)
    for (long long T : tiles) check(T, G);
  // tile_div on both sides of 2^32 - 1
  const long long as[] = {0, 1, 12345, 0xFFFFFFFELL, 0xFFFFFFFFLL, 0x100000000LL, 0x3FFFFFFFFFLL};
  const long long bs[] = {1, 3, 1104, 65536, 4000000};
  for (long long a : as)
    for (long long b : bs)
      if (ctd::tile_div(a, b) != a / b) fail("tile_div", a, 0, b, ctd::tile_div(a, b));
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("tile split ok\n");
  return 0;
}
