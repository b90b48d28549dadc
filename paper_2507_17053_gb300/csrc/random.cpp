// The seeded input generator of the benchmark workloads (the paper names no
// generator for "x ~ U(-1,1) from seed s"; this is the library's convention,
// shared with the Python workload descriptions so that a C caller can
// reproduce every input vector bit for bit).
//
// Counter-based splitmix64 (Steele, Lea, Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): value k of stream `seed` is
// the published splitmix64 finaliser applied to seed + (k + 1) * golden
// gamma (mod 2^64).  U(-1, 1): u = (z >> 11) * 2^-53 in [0, 1), value 2u - 1.
// N(0, 1): Box--Muller on the uniform pair (u_2k, u_2k+1), cosine branch,
// sqrt(-2 log1p(-u_2k)) cos(2 pi u_2k+1), with the C library's log1p and cos.
// Compiled without fused multiply-adds (-ffp-contract=off) so that every
// platform rounds the same way.
#include <cmath>
#include <cstdint>

#include "sbm.h"
#include "internal.hpp"

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kMix1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kMix2 = 0x94D049BB133111EBull;
constexpr double kPi = 3.14159265358979323846;

inline uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * kGamma;
  z = (z ^ (z >> 30)) * kMix1;
  z = (z ^ (z >> 27)) * kMix2;
  return z ^ (z >> 31);
}

inline double unit53(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

extern "C" int sbm_fill_random(int64_t n, uint64_t seed, uint64_t offset, int dist,
                               double* out_host) {
  if (n < 0 || (n > 0 && !out_host))
    return sbm::sbm_fail_detail(SBM_ERR_ARG, "n < 0 or NULL output");
  if (dist == SBM_DIST_UNIFORM) {
    for (int64_t i = 0; i < n; ++i)
      out_host[i] = 2.0 * unit53(splitmix64_at(seed, offset + (uint64_t)i)) - 1.0;
    return SBM_OK;
  }
  if (dist == SBM_DIST_NORMAL) {
    for (int64_t i = 0; i < n; ++i) {
      const uint64_t k = 2 * (offset + (uint64_t)i);
      const double u1 = unit53(splitmix64_at(seed, k));
      const double u2 = unit53(splitmix64_at(seed, k + 1));
      out_host[i] = std::sqrt(-2.0 * std::log1p(-u1)) * std::cos(2.0 * kPi * u2);
    }
    return SBM_OK;
  }
  return sbm::sbm_fail_detail(SBM_ERR_ARG, "unknown distribution");
}
