// Host checks of two index tables of the step kernel:
//  * tc_img_index (tensor-core contraction): per 128-row block and 16-wide K step one image
//    of 128 x 16 BF16 per term of the split (1 to 3).  The map must be a bijection onto the images, and inside an
//    image it must be the canonical K-major layout without swizzle that the shared-memory
//    descriptors declare: 8 x 8 core matrices with rows 16 bytes apart, the second core
//    matrix along K 128 bytes after the first (leading byte offset) and the next group of 8
//    rows 256 bytes after (stride byte offset).
//  * the separated form's multiset table: entry q packs m1 <= m2 <= m3 and the number of
//    distinct orderings; the first C(M + 2, 3) entries must be exactly the multisets of
//    indices below M for every M up to the table's mode limit, each once, with orderings
//    3! / (multiplicities!), which sum to M^3.
// Prints one line per failure and exits 1 if there is any.
#include "ctd_step.cuh"

#include <cstdio>
#include <vector>

static int failures = 0;

static void fail(const char* what, long long a, long long b, long long c) {
  if (failures < 20) std::printf("FAIL %s %lld %lld %lld\n", what, a, b, c);
  ++failures;
}

static void check_images(int nrb, int KS, int nimg) {
  using namespace ctd;
  const size_t total = static_cast<size_t>(nrb) * KS * nimg * kTcImgElems;
  std::vector<int> seen(total, 0);
  for (long long i = 0; i < 128LL * nrb; ++i)
    for (int k = 0; k < 16 * KS; ++k)
      for (int h = 0; h < nimg; ++h) {
        const size_t idx = tc_img_index(i, k, h, KS, nimg);
        if (idx >= total) {
          fail("range", i, k, static_cast<long long>(idx));
          continue;
        }
        ++seen[idx];
        // image of (row block, K step, BF16 term), then the byte offset inside it
        const size_t img = static_cast<size_t>(((i >> 7) * KS + (k >> 4)) * nimg + h);
        const long long off = 2LL * static_cast<long long>(idx - img * kTcImgElems);
        const int r = static_cast<int>(i & 127), kk = k & 15;
        const long long want = (r >> 3) * 256LL + (kk >> 3) * 128LL + (r & 7) * 16LL + (kk & 7) * 2LL;
        if (off != want) fail("layout", i, k, off);
      }
  for (size_t e = 0; e < total; ++e)
    if (seen[e] != 1) fail("bijection", nrb, KS, static_cast<long long>(e));
}

static void check_sep_table() {
  using namespace ctd;
  const SepTable t = make_sep_table();
  if (sep_terms(kMaxSepModes) != kMaxSep) fail("size", sep_terms(kMaxSepModes), kMaxSep, 0);
  for (int M = 0; M <= kMaxSepModes; ++M) {
    std::vector<int> count(static_cast<size_t>(M) * M * M, 0);
    long long orderings = 0;
    for (int q = 0; q < sep_terms(M); ++q) {
      const unsigned e = t.e[q];
      const int m1 = e & 0xFF, m2 = (e >> 8) & 0xFF, m3 = (e >> 16) & 0xFF, ord = e >> 24;
      if (!(m1 <= m2 && m2 <= m3 && m3 < M)) {
        fail("multiset", M, q, e);
        continue;
      }
      ++count[(static_cast<size_t>(m1) * M + m2) * M + m3];
      const int want = (m1 == m3) ? 1 : ((m1 == m2 || m2 == m3) ? 3 : 6);
      if (ord != want) fail("orderings", M, q, ord);
      orderings += ord;
    }
    for (int m1 = 0; m1 < M; ++m1)
      for (int m2 = m1; m2 < M; ++m2)
        for (int m3 = m2; m3 < M; ++m3)
          if (count[(static_cast<size_t>(m1) * M + m2) * M + m3] != 1) fail("once", M, m1 * 256 + m2, m3);
    if (orderings != static_cast<long long>(M) * M * M) fail("M^3", M, orderings, 0);
  }
}

int main() {
  const int blocks[] = {1, 2, 3};
  const int ksteps[] = {1, 2, 3, 5};
  for (int nrb : blocks)
    for (int KS : ksteps)
      for (int nimg = 1; nimg <= 3; ++nimg) check_images(nrb, KS, nimg);
  // the products of the tensor-core precisions: every pair of term orders summing to at most
  // nimg - 1, each once, the leading product first
  using namespace ctd;
  for (int nimg = 1; nimg <= 3; ++nimg) {
    int seen[3][3] = {};
    for (int p = 0; p < tc_npairs(nimg); ++p) {
      const int a = tc_pair_a(p), b = tc_pair_b(p);
      if (a + b > nimg - 1) fail("pair order", nimg, a, b);
      ++seen[a][b];
    }
    for (int a = 0; a < nimg; ++a)
      for (int b = 0; a + b < nimg; ++b)
        if (seen[a][b] != 1) fail("pair", nimg, a, b);
  }
  check_sep_table();
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("layout ok\n");
  return 0;
}
