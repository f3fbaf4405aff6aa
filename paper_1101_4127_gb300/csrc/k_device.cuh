// k_device.cuh -- device building blocks of the transport kernels:
// counter-based random numbers, isotropic directions, exp(-tau) and the box
// lookup of a packet or a cell.  Every routine here is specified down to the
// order of its floating-point operations so that the FP64 form reproduces
// the FP64 specification bit for bit (the translation units that include it
// for the FP64 form are compiled with -fmad=false).
#pragma once
#include <stdint.h>

#include "crash_internal.cuh"

namespace crash {

// ---------------------------------------------------------------- Philox
// Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of two
// 32x32->64 multiplications whose high halves are xored with the other two
// counter words and the round key; the key advances by the golden-ratio and
// sqrt(3)-1 Weyl increments.
struct PhiloxKey { uint32_t k0, k1; };

__device__ __forceinline__ uint4 philox_round(uint4 c, PhiloxKey k) {
  const uint32_t mA = 0xD2511F53u, mB = 0xCD9E8D57u;
  uint32_t hiA = __umulhi(mA, c.x), loA = mA * c.x;
  uint32_t hiB = __umulhi(mB, c.z), loB = mB * c.z;
  return make_uint4(hiB ^ c.y ^ k.k0, loB, hiA ^ c.w ^ k.k1, loA);
}

__device__ __forceinline__ uint4 philox10(uint4 ctr, uint64_t seed) {
  PhiloxKey k{(uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32)};
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    ctr = philox_round(ctr, k);
    k.k0 += 0x9E3779B9u;
    k.k1 += 0xBB67AE85u;
  }
  return ctr;
}

// 53-bit uniform in [0, 1) from two 32-bit words (hi word more significant)
__device__ __forceinline__ double uniform53(uint32_t lo, uint32_t hi) {
  unsigned long long w = ((unsigned long long)hi << 32) | (unsigned long long)lo;
  return (double)(w >> 11) * 1.1102230246251565404236316680908203125e-16;  // 2^-53
}

// Isotropic unit vector by Marsaglia's rejection (Ann. Math. Stat. 1972):
// (v1, v2) uniform on [-1,1)^2 accepted when 0 < s = v1^2 + v2^2 < 1, then
// (2 v1 sqrt(1-s), 2 v2 sqrt(1-s), 1 - 2s).  Attempt a draws Philox counter
// (pkt, src, step, a).  Returns false after 64 rejected attempts.
__device__ __forceinline__ bool iso_direction(uint64_t seed, uint32_t step, uint32_t src,
                                              uint32_t pkt, double& dx, double& dy, double& dz) {
  for (uint32_t a = 0; a < 64u; ++a) {
    uint4 r = philox10(make_uint4(pkt, src, step, a), seed);
    double v1 = 2.0 * uniform53(r.x, r.y) - 1.0;
    double v2 = 2.0 * uniform53(r.z, r.w) - 1.0;
    double s = v1 * v1 + v2 * v2;
    if (s < 1.0 && s != 0.0) {
      double root = sqrt(1.0 - s);
      dx = (2.0 * v1) * root;
      dy = (2.0 * v2) * root;
      dz = 1.0 - 2.0 * s;
      return true;
    }
  }
  return false;
}

// The same draws with the acceptance test in FP64 (so that every packet
// takes the same attempt as in the FP64 form) and the direction in FP32.
__device__ __forceinline__ bool iso_direction_f32(uint64_t seed, uint32_t step, uint32_t src,
                                                  uint32_t pkt, float& dx, float& dy, float& dz) {
  for (uint32_t a = 0; a < 64u; ++a) {
    uint4 r = philox10(make_uint4(pkt, src, step, a), seed);
    double v1 = 2.0 * uniform53(r.x, r.y) - 1.0;
    double v2 = 2.0 * uniform53(r.z, r.w) - 1.0;
    double s = v1 * v1 + v2 * v2;
    if (s < 1.0 && s != 0.0) {
      const float sf = (float)s;
      const float root = sqrtf(1.0f - sf);
      dx = (2.0f * (float)v1) * root;
      dy = (2.0f * (float)v2) * root;
      dz = 1.0f - 2.0f * sf;
      return true;
    }
  }
  return false;
}

// Start of the re-emission packet of a cell (diffuse recombination field):
// the offsets (in cells) of a point drawn uniformly in the cell.  The
// packet uses the Philox counters of a source 0x80000000 | (cell >> 32) and
// packet cell & 0xffffffff (cell: index within its box), so no point source
// shares them; its direction takes attempts 0..63 as for a source packet,
// the offsets attempts 64 (x, y) and 65 (z), each the top 31 bits of a
// 64-bit word times 2^-31 (cell + offset is exact in FP64 and below the
// next cell).
__device__ __forceinline__ double uniform31(uint32_t lo, uint32_t hi) {
  unsigned long long w = ((unsigned long long)hi << 32) | (unsigned long long)lo;
  return (double)(w >> 33) * 4.656612873077392578125e-10;   // 2^-31
}
__device__ __forceinline__ uint32_t rec_src_id(int64_t cell) {
  return 0x80000000u | (uint32_t)((unsigned long long)cell >> 32);
}
__device__ __forceinline__ void rec_offsets(uint64_t seed, uint32_t step, int64_t cell, double& ox,
                                            double& oy, double& oz) {
  const uint32_t src = rec_src_id(cell), pkt = (uint32_t)cell;
  const uint4 r0 = philox10(make_uint4(pkt, src, step, 64u), seed);
  const uint4 r1 = philox10(make_uint4(pkt, src, step, 65u), seed);
  ox = uniform31(r0.x, r0.y);
  oy = uniform31(r0.z, r0.w);
  oz = uniform31(r1.x, r1.y);
}

// ------------------------------------------------------ space-filling keys
// Key of bucket (x, y, z), each coordinate below 2^b, along a space-filling
// curve of 2^(3b) positions: the Morton (Z) order interleaves the bits, x
// least significant; the Hilbert order first maps the coordinates to the
// curve's transposed index by Skilling's transform (AIP Conf. Proc. 707,
// 2004: undo the excess rotations and reflections level by level, then
// Gray-encode) and interleaves that, x most significant.  Consecutive
// Hilbert keys are face neighbours; consecutive Morton keys may jump.
__host__ __device__ __forceinline__ unsigned spread_bits3(unsigned v) {   // 10 bits -> every third bit
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__host__ __device__ __forceinline__ unsigned curve_key3(unsigned x, unsigned y, unsigned z, int b,
                                                        bool hilbert) {
  if (!hilbert) return spread_bits3(x) | (spread_bits3(y) << 1) | (spread_bits3(z) << 2);
  if (b <= 0) return 0u;
  unsigned X0 = x, X1 = y, X2 = z;
  const unsigned M = 1u << (b - 1);
  for (unsigned Q = M; Q > 1u; Q >>= 1) {
    const unsigned P = Q - 1u;
    // axis 0: invert the low bits when its Q bit is set
    if (X0 & Q) X0 ^= P;
    // axes 1, 2: invert axis 0's low bits, or exchange them with axis i's
    if (X1 & Q) {
      X0 ^= P;
    } else {
      const unsigned t = (X0 ^ X1) & P;
      X0 ^= t;
      X1 ^= t;
    }
    if (X2 & Q) {
      X0 ^= P;
    } else {
      const unsigned t = (X0 ^ X2) & P;
      X0 ^= t;
      X2 ^= t;
    }
  }
  X1 ^= X0;
  X2 ^= X1;
  unsigned t = 0;
  for (unsigned Q = M; Q > 1u; Q >>= 1)
    if (X2 & Q) t ^= Q - 1u;
  X0 ^= t;
  X1 ^= t;
  X2 ^= t;
  return (spread_bits3(X0) << 2) | (spread_bits3(X1) << 1) | spread_bits3(X2);
}

// ---------------------------------------------------------------- exp(-tau)
// e^-tau, tau >= 0: split -tau = k ln2 + r (Cody & Waite 1980 two-constant
// reduction, ln2 high part with 40 significant bits), e^r by its degree-13
// Taylor polynomial in Horner order, scaled by 2^k.  tau above 50 returns 0
// (no count below 2^63 keeps a transmitted photon there).
__device__ __forceinline__ double exp_neg_spec(double tau) {
  if (!(tau <= 50.0)) return 0.0;
  const double x = -tau;
  const double kf = rint(x * 0x1.71547652b82fep+0);
  const double r = (x - kf * 0x1.62e42fefa2000p-1) - kf * 0x1.9ef35793c7673p-41;
  double p = 0x1.6124613a86d09p-33;      // 1/13!
  p = p * r + 0x1.1eed8eff8d898p-29;     // 1/12!
  p = p * r + 0x1.ae64567f544e4p-26;     // 1/11!
  p = p * r + 0x1.27e4fb7789f5cp-22;     // 1/10!
  p = p * r + 0x1.71de3a556c734p-19;     // 1/9!
  p = p * r + 0x1.a01a01a01a01ap-16;     // 1/8!
  p = p * r + 0x1.a01a01a01a01ap-13;     // 1/7!
  p = p * r + 0x1.6c16c16c16c17p-10;     // 1/6!
  p = p * r + 0x1.1111111111111p-7;      // 1/5!
  p = p * r + 0x1.5555555555555p-5;      // 1/4!
  p = p * r + 0x1.5555555555555p-3;      // 1/3!
  p = p * r + 0.5;
  p = p * r + 1.0;
  p = p * r + 1.0;
  return ldexp(p, (int)kf);
}

// ceil(log2 x) for x > 0, exact
__device__ __forceinline__ int ceil_log2_dev(double x) {
  int e;
  double m = frexp(x, &e);
  return (m == 0.5) ? e - 1 : e;
}

// ---------------------------------------------------------------- lookups
// index of the last box with key(box) <= v (boxes sorted by key)
__device__ __forceinline__ int box_of_packet(const BoxMeta* b, int n, int64_t gid) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b[mid].pkt_off <= gid) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int box_of_cell(const BoxMeta* b, int n, int64_t cell) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b[mid].cell_off <= cell) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}

}  // namespace crash
