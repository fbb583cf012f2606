// Warp-wide multi-limb additions: limb l of a number sits in lane l % 32 of chunk l / 32;
// the one-bit carries between lanes are resolved with generate/propagate ballots.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bs {

// x + y + (carry into this lane); cin is the carry into the chunk, updated to the carry
// out of it
__device__ __forceinline__ uint32_t ballot_add(uint32_t x, uint32_t y, uint32_t& cin, int lane) {
  const uint32_t s = x + y;
  const uint32_t G = __ballot_sync(0xffffffffu, s < x);
  const uint32_t Pm = __ballot_sync(0xffffffffu, s == 0xffffffffu) & ~G;
  const uint32_t X = G | Pm;
  const uint64_t S = (uint64_t)X + G + cin;
  const uint32_t C = (uint32_t)S ^ X ^ G;
  cin = (uint32_t)(S >> 32);
  return s + ((C >> lane) & 1u);
}

// x - y - (borrow into this lane); bin is the borrow into the chunk, updated
__device__ __forceinline__ uint32_t ballot_sub(uint32_t x, uint32_t y, uint32_t& bin, int lane) {
  const uint32_t d = x - y;
  const uint32_t G = __ballot_sync(0xffffffffu, x < y);            // generates a borrow
  const uint32_t Pm = __ballot_sync(0xffffffffu, d == 0u) & ~G;   // propagates one
  const uint32_t X = G | Pm;
  const uint64_t S = (uint64_t)X + G + bin;
  const uint32_t C = (uint32_t)S ^ X ^ G;
  bin = (uint32_t)(S >> 32);
  return d - ((C >> lane) & 1u);
}

}  // namespace bs
