// Correctly rounded FP64 operations on the integer pipes.
//
// The recovery needs three floating-point operations per edge or vertex, each
// rounded once to nearest-even as IEEE 754 defines them:
//   r = fl(1/w)            step A1, the resistive weight of a tree edge (Eq. RT)
//   R = fl(D * 2^-S)       step A3, the exact fixed-point path sum to FP64
//   s = fl(w * R)          step A3, the stretch score (one hardware multiply)
// On this GPU the double-precision pipe is a small fraction of the integer and
// single-precision pipes; the reciprocal (a multi-step sequence on that pipe)
// and the conversion (which has no single hardware instruction) are computed
// from the bit patterns with integer arithmetic.  The results are bit-identical
// to the IEEE operations (the test-suite compares them with the oracle's C
// doubles); inputs outside the normal range of the fast path fall back to the
// hardware operation.
//
//   reciprocal: Newton's iteration x <- x + x (1 - m x) for 1/m on the 53-bit
//     significand m, started from the single-precision reciprocal of its top
//     24 bits and run twice in 128-bit fixed point (each step squares the
//     relative error: 2^-22 -> 2^-44 -> below one unit), then the exact
//     quotient floor(2^105 / m) by comparing products, and the rounding bit
//     from the remainder (no ties: 2^106 / m is never an odd integer for a
//     significand that is not a power of two).
//   fixed point to FP64: the leading bit of the integer fixes the exponent;
//     the 53 bits below it, rounded by the remainder, the significand.
#pragma once

#include <stdint.h>

namespace pdg {

typedef unsigned __int128 u128;

#ifdef __CUDACC__
#define PDG_HD __host__ __device__ __forceinline__
#else
#define PDG_HD inline
#endif

constexpr uint64_t kMant = (1ull << 52) - 1;

PDG_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

PDG_HD float rcp_f32(float f) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(f);
#else
  return 1.0f / f;
#endif
}

// round(2^105 / m) for a significand 2^52 < m < 2^53; *ok is false if the
// bounded correction did not settle (it always does; the caller then falls
// back to a hardware division)
PDG_HD uint64_t rcp_significand(uint64_t m, bool* ok) {
  const u128 two105 = (u128)1 << 105;
  // 2^29 / m to about 2^-22 relative, as 2^105 / m in fixed point
  const float y = rcp_f32((float)(uint32_t)(m >> 29));
  uint64_t x = (uint64_t)(y * 0x1p76f);  // y * 2^76, truncated
#pragma unroll
  for (int it = 0; it < 2; it++) {
    const u128 mx = (u128)m * x;
    const bool above = mx > two105;
    const u128 e = above ? mx - two105 : two105 - mx;  // |2^105 - m x| < 2^86
    const u128 t = (u128)(uint64_t)(e >> 33) * x;        // e x / 2^33
    const uint64_t c = (uint64_t)(t >> 72);              // e x / 2^105
    x = above ? x - c : x + c;
  }
  u128 mx = (u128)m * x;
  bool settled = false;
  for (int k = 0; k < 8; k++) {  // x = floor(2^105 / m): m x <= 2^105 < m (x + 1)
    if (mx > two105) {
      x--;
      mx -= m;
    } else if (two105 - mx >= m) {
      x++;
      mx += m;
    } else {
      settled = true;
      break;
    }
  }
  *ok = settled;
  const uint64_t rem = (uint64_t)(two105 - mx);
  return (rem > m - rem) ? x + 1 : x;  // 2 rem > m: round up
}

// IEEE bits of fl(1/w) for positive normal w whose reciprocal is normal;
// *ok is false when the caller must use a hardware division instead
PDG_HD uint64_t rcp_rn_bits(uint64_t wb, bool* ok) {
  const uint64_t e = wb >> 52;  // biased exponent (sign bit 0)
  const uint64_t f = wb & kMant;
  *ok = (e >= 1 && e <= 2044);
  if (f == 0) return (2046 - e) << 52;  // 1 / 2^(e-1023) exactly
  const uint64_t q = rcp_significand(f | (1ull << 52), ok);
  return ((2045 - e) << 52) | (q & kMant);  // q in (2^52, 2^53): 1/w = q 2^(1022 - (e-1023) - 52 - 52)
}

// IEEE bits of fl(x * 2^-S) for an integer 0 < x = hi 2^64 + lo < 2^115 (the
// exact path sums stay below 2^97) whose value is a normal double: every shift
// and mask stays within 64 bits.
PDG_HD uint64_t fixed_hl_to_bits(uint64_t hi, uint64_t lo, int S) {
  int p = hi ? 127 - clz64(hi) : 63 - clz64(lo);  // leading bit
  const int sh = p - 52;                          // at most 62
  uint64_t q;
  if (sh <= 0) {
    q = lo << (-sh);  // exact (hi is zero here)
  } else {
    q = (hi << (64 - sh)) | (lo >> sh);  // below 2^53: hi < 2^(p - 63)
    const uint64_t rem = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) {
      q++;
      if (q >> 53) {
        q >>= 1;
        p++;
      }
    }
  }
  return ((uint64_t)(p - S + 1023) << 52) | (q & kMant);
}

}  // namespace pdg
