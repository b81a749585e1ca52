// 32-bit modular arithmetic on the device for primes 2^30 < p < 2^31.
//
// Residues live in [0, p).  Multiplication is Montgomery's REDC with
// R = 2^32 in its signed form: for x < p * 2^32, m = x_lo * p^-1 mod 2^32
// makes x - m p divisible by 2^32 with the low words cancelling exactly, so
// x / R mod p = x_hi - umulhi(m, p), a value in (-p, p) that one unsigned
// min() folds into [0, p).  Because 2p < 2^32, a sum of two products of
// residues stays below p * 2^32 and needs a single REDC (the fused
// a*b - c*d of the elimination update).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define PD_HD __host__ __device__ __forceinline__
#define PD_D __device__ __forceinline__

struct ModP {
  uint32_t p;     // the prime
  uint32_t pinv;  // p^-1 mod 2^32
  uint32_t r1;    // R mod p      (Montgomery form of 1)
  uint32_t r2;    // R^2 mod p    (to enter Montgomery form)
};

PD_D uint32_t redc(uint64_t x, uint32_t p, uint32_t pinv) {
  uint32_t lo = (uint32_t)x;
  uint32_t hi = (uint32_t)(x >> 32);
  uint32_t m = lo * pinv;
  uint32_t r = hi - __umulhi(m, p);
  return min(r, r + p);
}

// a * b / R mod p, valid for a * b < p * 2^32 (e.g. a < 2^32, b < p).
PD_D uint32_t mmul(uint32_t a, uint32_t b, uint32_t p, uint32_t pinv) {
  return redc((uint64_t)a * b, p, pinv);
}

// (a*b - c*d) / R mod p for a, b, c, d in [0, p).
PD_D uint32_t mfms(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t p,
                   uint32_t pinv) {
  return redc((uint64_t)a * b + (uint64_t)c * (p - d), p, pinv);
}

// Largest prime for mfms3: with x <= 3 (p-1)^2 the REDC value lies in
// (-p, r_max], r_max = floor(3 (p-1)^2 / 2^32), and two folds bring it to
// [0, p) exactly when r_max + p < 2^32 and r_max < 2p.
#define PD_FOLD3_MAX 1865126253u

// x / R mod p for x < 3 p^2 (a sum of up to three products of residues) and
// p <= PD_FOLD3_MAX: one REDC leaves r in (-p, r_max] (an interval shorter
// than 2^32, so no two values share a 32-bit pattern); min(r, r + p) folds
// the wrapped negatives into [0, p), then min(r, r - p) folds [p, r_max]
// (r_max < 2p) into [0, p).  mfms3: (a*b + c*d + e*f) / R mod p for all six
// operands in [0, p).
PD_D uint32_t redc3(uint64_t x, uint32_t p, uint32_t pinv) {  // x < 3 p^2, p <= PD_FOLD3_MAX
  const uint32_t m = (uint32_t)x * pinv;
  uint32_t r = (uint32_t)(x >> 32) - __umulhi(m, p);
  r = min(r, r + p);
  return min(r, r - p);
}

// x / R mod p for x < 4 p^2 (a sum of up to four products of residues) and
// any p < 2^31: with hi = floor(x / 2^32) < 4 p^2 / 2^32 < 2p and
// mh = umulhi(m, p) < p, the REDC value hi - mh lies in (-p, 2p); its sign is
// hi < mh, after which one conditional subtraction reaches [0, p).
PD_D uint32_t redc4(uint64_t x, uint32_t p, uint32_t pinv) {
  const uint32_t m = (uint32_t)x * pinv;
  const uint32_t hi = (uint32_t)(x >> 32), mh = __umulhi(m, p);
  uint32_t r = hi - mh;
  r = (hi < mh) ? r + p : r;
  return min(r, r - p);
}

PD_D uint32_t mfms3(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e, uint32_t f,
                    uint32_t p, uint32_t pinv) {
  return redc3((uint64_t)a * b + (uint64_t)c * d + (uint64_t)e * f, p, pinv);
}

PD_D uint32_t addm(uint32_t a, uint32_t b, uint32_t p) {
  uint32_t s = a + b;
  return min(s, s - p);
}

PD_D uint32_t subm(uint32_t a, uint32_t b, uint32_t p) {
  uint32_t d = a - b;
  return min(d, d + p);
}

// Montgomery-form power: returns (x/R)^e in Montgomery form, x in Montgomery
// form; `one` is R mod p.
PD_D uint32_t mpow(uint32_t x, uint32_t e, uint32_t one, uint32_t p, uint32_t pinv) {
  uint32_t r = one;
  while (e) {
    if (e & 1u) r = mmul(r, x, p, pinv);
    x = mmul(x, x, p, pinv);
    e >>= 1;
  }
  return r;
}

// Reduce a signed 32-bit coefficient into [0, p) (p > 2^30 so at most two
// corrections each way).
PD_D uint32_t reduce_i32(int32_t c, uint32_t p) {
  int64_t t = c;
  if (t < 0) t += p;
  if (t < 0) t += p;
  if (t >= (int64_t)p) t -= p;
  return (uint32_t)t;
}

