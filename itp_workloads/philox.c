/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11),
 * the integer part of the seeded input generator in itp_workloads, written in
 * C for speed.  Produces the same uniforms as the numpy version: for
 * counters (c0 = first + t, c1, c2, c3) and key (k0, k1), out[2t] and
 * out[2t+1] are the two 53-bit uniforms (hi word >> 5, lo word >> 6) built
 * from words (0,1) and (2,3).  Plain C, no intrinsics. */
#include <stdint.h>

static void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    if (r < 9) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
}

static double u53(uint32_t hi, uint32_t lo) {
  return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6) + 0.5) / 9007199254740992.0;
}

void philox_uniform_pairs(uint64_t count, uint32_t first, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t k0, uint32_t k1, double* out) {
  for (uint64_t t = 0; t < count; ++t) {
    uint32_t c[4] = {first + (uint32_t)t, c1, c2, c3};
    philox10(c, k0, k1);
    out[2 * t] = u53(c[0], c[1]);
    out[2 * t + 1] = u53(c[2], c[3]);
  }
}
