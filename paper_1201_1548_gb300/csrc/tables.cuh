// Host prime table and per-context device tables.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace bs {

struct HostPrimes {
  std::vector<uint32_t> p;          // the table: two decreasing runs (3p < 2^32 first)
  int n_small = 0;                  // length of the first run
  std::vector<PrimeConst> pc;       // constants per prime
  std::vector<uint32_t> pw, mpw;    // [T][kMaxLimbs + 1]
  std::vector<int64_t> lg_prefix;   // [T + 1]
};

// built once per process
const HostPrimes& host_primes();
// position of p in the table, -1 if p is not a table prime
int table_index(uint32_t p);

struct DeviceTables {
  PrimeConst* pc = nullptr;
  uint32_t* pw = nullptr;
  uint32_t* mpw = nullptr;
  int64_t* lgp = nullptr;
  uint32_t *tw = nullptr, *itw = nullptr, *cp = nullptr, *icp = nullptr, *ninv = nullptr;
  uint32_t *twp = nullptr, *itwp = nullptr, *tws = nullptr;
  uint32_t* ginv = nullptr;
  uint32_t* pp = nullptr;
  int LPP = 0;
  uint32_t* ws_m = nullptr;
  int64_t* ws_moff = nullptr;
  uint32_t* ws_y = nullptr;
  int32_t* ws_yoff = nullptr;
  uint32_t* q62 = nullptr;
  int64_t ws_m_words = 0;
  int WK = 0;
  int T = 0, Tt = 0, NT = 0, logNT = 0, Tg = 0;
  int generation = 0;

  int init(cudaStream_t s);
  // make transform and Garner tables cover the first needT primes and sizes up to
  // 2^needLogN; grows geometrically; synchronises the stream when it grows
  int ensure(int needT, int needLogN, cudaStream_t s);
  void release();
  Tables view() const;
};

}  // namespace bs
