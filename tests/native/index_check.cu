// Host-side check of the index arithmetic the kernels use (run by
// tests/test_index_cpu.py; no GPU needed).
//
//  * site_index (hsg_device.cuh): for every site of both colours, its own
//    colour-split index q, its six neighbours' indices and its Philox site
//    number, against plain coordinate arithmetic with periodic wrap -- every
//    neighbour of the right colour, inside [0, N/2), at the right place.
//    All sites for L = 4 ... 96 and 128, 256; sampled sites at L = 1624 (the
//    largest accepted side, indices near the 32-bit limits).
//  * fast_div / make_fastdiv (the pool kernels' multiply-shift division):
//    against n / d for every divisor the pools use (L/2 and L * L/2 for even
//    L <= 1624) at edge and random 32-bit n.
// Prints "ok" and returns 0, or prints the first mismatch and returns 1.
#include <cstdint>
#include <cstdio>
#include <random>

#include "hsg_device.cuh"

namespace {

int failures = 0;

void fail(const char* what, long long L, long long a, long long b, long long c) {
  if (failures++ < 10) std::printf("FAIL %s L=%lld: %lld %lld %lld\n", what, L, a, b, c);
}

// Colour-split index of site (x, y, z) of an L lattice, from coordinates.
uint32_t cs_index(uint32_t x, uint32_t y, uint32_t z, uint32_t L) { return (z * L + y) * (L / 2) + (x >> 1); }

void check_site(uint32_t L, uint32_t colour, uint32_t xh, uint32_t y, uint32_t z) {
  const uint32_t Lh = L / 2;
  const hsg::SiteIndex ix = hsg::site_index(xh, y, z, L, Lh, colour);
  const uint32_t p = (colour + y + z) & 1u;
  const uint32_t x = 2 * xh + p;
  const unsigned long long nh = (unsigned long long)L * L * Lh;
  if ((x + y + z) % 2 != colour) fail("colour of x", L, x, y, z);
  if (ix.q != cs_index(x, y, z, L) || ix.q >= nh) fail("own index", L, x, y, z);
  if ((unsigned long long)ix.site != (unsigned long long)x + (unsigned long long)y * L + (unsigned long long)z * L * L)
    fail("site number", L, x, y, z);
  const uint32_t nb[6][3] = {{(x + 1) % L, y, z}, {(x + L - 1) % L, y, z}, {x, (y + 1) % L, z},
                             {x, (y + L - 1) % L, z}, {x, y, (z + 1) % L}, {x, y, (z + L - 1) % L}};
  const uint32_t got[6] = {ix.q_xp, ix.q_xm, ix.q_yp, ix.q_ym, ix.q_zp, ix.q_zm};
  for (int k = 0; k < 6; ++k) {
    const uint32_t nx = nb[k][0], ny = nb[k][1], nz = nb[k][2];
    if ((nx + ny + nz) % 2 == colour) fail("neighbour colour", L, x, y, k);
    if (got[k] >= nh || got[k] != cs_index(nx, ny, nz, L)) fail("neighbour index", L, x, y, k);
  }
}

void check_lattice_full(uint32_t L) {
  for (uint32_t c = 0; c < 2; ++c)
    for (uint32_t z = 0; z < L; ++z)
      for (uint32_t y = 0; y < L; ++y)
        for (uint32_t xh = 0; xh < L / 2; ++xh) check_site(L, c, xh, y, z);
}

void check_lattice_sampled(uint32_t L, std::mt19937_64& rng) {
  const uint32_t e[] = {0u, 1u, L / 2 - 1, L - 2, L - 1};
  for (uint32_t c = 0; c < 2; ++c)
    for (uint32_t a : e)
      for (uint32_t b : e)
        for (uint32_t d : e) check_site(L, c, a % (L / 2), b, d);
  std::uniform_int_distribution<uint32_t> u(0, L - 1), uh(0, L / 2 - 1);
  for (int k = 0; k < 1000000; ++k) check_site(L, k & 1, uh(rng), u(rng), u(rng));
}

void check_fastdiv(uint32_t d, std::mt19937_64& rng) {
  const hsg::FastDiv f = hsg::make_fastdiv(d);
  const uint64_t edges[] = {0, 1, d - 1ull, d, d + 1ull, 2ull * d - 1, 2ull * d, 0x7FFFFFFFull, 0x80000000ull,
                            0xFFFFFFFEull, 0xFFFFFFFFull, (0xFFFFFFFFull / d) * d, (0xFFFFFFFFull / d) * d - 1};
  for (uint64_t n64 : edges) {
    if (n64 > 0xFFFFFFFFull) continue;
    const uint32_t n = (uint32_t)n64;
    if (hsg::fast_div(n, f) != n / d) fail("fast_div", d, n, hsg::fast_div(n, f), n / d);
  }
  std::uniform_int_distribution<uint32_t> u;
  for (int k = 0; k < 2000; ++k) {
    const uint32_t n = u(rng);
    if (hsg::fast_div(n, f) != n / d) fail("fast_div", d, n, hsg::fast_div(n, f), n / d);
  }
}

}  // namespace

int main() {
  std::mt19937_64 rng(1006);
  for (uint32_t L = 4; L <= 96; L += 2) check_lattice_full(L);
  check_lattice_full(128);
  check_lattice_full(256);
  check_lattice_sampled(1624, rng);
  for (uint32_t L = 4; L <= 1624; L += 2) {
    check_fastdiv(L / 2, rng);
    check_fastdiv(L * (L / 2), rng);
  }
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
