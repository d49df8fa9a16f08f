// sround.cuh -- stochastically rounded FP16 stores, shared by the step
// kernels that use them (the F16R form, and the F16S form with stochastic
// rounding).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace clbm {

// Stochastic rounding of the stores: a value is rounded up in magnitude with
// probability equal to the fraction of an FP16 ulp it carries, so increments
// far below one ulp (a weak body force, a slow transient) survive on average
// instead of being rounded away every step.  The random bits depend only on
// the node index, the direction pair and the lattice's own step count, so a
// lattice gives the same result alone and in a batch: one integer hash of
// (node, step) (the finaliser of MurmurHash3), then one step per pair of
// directions of a 32-bit linear congruential generator with the multiplier
// and increment of PCG (O'Neill, 2014).
__device__ __forceinline__ uint32_t sr_seed(uint32_t node, uint32_t step) {
  uint32_t h = node ^ (step * 0x9E3779B9u);
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Two values at once with the GB300's stochastic-rounding conversion
// (cvt.rs.f16x2.f32: each value rounded up in magnitude with the probability
// of the fraction of an FP16 ulp it carries).  hi receives a, lo b; the
// conversion adds the low 13 bits of each 16-bit half of the random word
// below the kept mantissa (measured: bits 0-12 round b, bits 16-28 round a).
// One 32-bit step of the generator above feeds both, with its upper half
// folded into the lower one: the low bits of a power-of-two-modulus LCG
// have short periods, its high bits do not.
__device__ __forceinline__ void enc16_sr2(float a, float b, uint32_t& state, __half& hi,
                                          __half& lo) {
  state = state * 747796405u + 2891336453u;
  const uint32_t rbits = state ^ (state >> 16);
  uint32_t d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;"
      : "=r"(d)
      : "f"(a), "f"(b), "r"(rbits));
  hi = __ushort_as_half(static_cast<unsigned short>(d >> 16));
  lo = __ushort_as_half(static_cast<unsigned short>(d & 0xFFFFu));
}

}  // namespace clbm
