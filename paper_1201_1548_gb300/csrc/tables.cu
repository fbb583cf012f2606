// The prime table and the per-context device tables.
//
// Prime table: every prime 2^30 < p < 2^31 with p = 1 (mod 2^14), in two decreasing runs
// (first those with 3p < 2^32),
// found with a deterministic Miller-Rabin test (bases 2, 7, 61 are sufficient below
// 4,759,123,141 -- G. Jaeschke, Math. Comp. 61 (1993)).  p = 1 mod 2^14 gives every prime
// a multiplicative subgroup of order 2^14, so each prime evaluates on a coset g * <omega>
// of up to 16384 points (g its smallest primitive root), which never contains 0, +1 or -1.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tables.cuh"

namespace bs {

static uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) { return (a * b) % m; }  // m < 2^32

static bool is_prime_u32(uint32_t n) {
  if (n < 2) return false;
  static const uint32_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (uint32_t q : small) {
    if (n == q) return true;
    if (n % q == 0) return false;
  }
  uint32_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (uint32_t a : {2u, 7u, 61u}) {
    if (a % n == 0) continue;
    uint64_t x = host_powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      x = mulmod64(x, x, n);
      if (x == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

// The representative c of each prime's evaluation coset c <omega>: c = g^e for the first e
// of E mod (p - 1), E mod (p - 1) + 2, ... (E = 0x9E3779B9, odd, so every e is odd) with
// c^(2^kLogNMax) != 1, i.e. c outside the subgroup of every transform size.  The smallest
// primitive root g itself would be a poor choice: it is a small integer (3 for many table
// primes), so x = g would be an evaluation point of every transform and a vertical
// asymptote there would reject the prime.
static uint32_t coset_rep(uint32_t p, uint32_t g) {
  const uint64_t pm1 = p - 1;
  uint64_t e = 0x9E3779B9ull % pm1;
  for (;;) {
    const uint32_t c = host_powmod(g, e, p);
    if (host_powmod(c, 1ull << kLogNMax, p) != 1u) return c;
    e = (e + 2) % pm1;
  }
}

static uint32_t primitive_root(uint32_t p) {
  std::vector<uint32_t> fs;
  uint32_t n = p - 1;
  for (uint32_t d = 2; (uint64_t)d * d <= n; d += (d == 2 ? 1 : 2)) {
    if (n % d == 0) {
      fs.push_back(d);
      while (n % d == 0) n /= d;
    }
  }
  if (n > 1) fs.push_back(n);
  for (uint32_t g = 2;; ++g) {
    bool ok = true;
    for (uint32_t q : fs)
      if (host_powmod(g, (p - 1) / q, p) == 1) {
        ok = false;
        break;
      }
    if (ok) return g;
  }
}

int table_index(uint32_t p) {
  const HostPrimes& H = host_primes();
  // each run is decreasing: binary search in the run p belongs to
  const auto lo = p <= kSmallPrimeMax ? H.p.begin() : H.p.begin() + H.n_small;
  const auto hi = p <= kSmallPrimeMax ? H.p.begin() + H.n_small : H.p.end();
  const auto it = std::lower_bound(lo, hi, p, std::greater<uint32_t>());
  return (it != hi && *it == p) ? (int)(it - H.p.begin()) : -1;
}

const HostPrimes& host_primes() {
  static HostPrimes H;
  static std::once_flag once;
  std::call_once(once, [] {
    // the primes p = 1 mod 2^kLogNMax with 2^30 < p < 2^31 in two runs, each decreasing:
    // first those with 3p < 2^32 (p <= kSmallPrimeMax), whose fused elimination updates
    // need no fold, then the rest
    const uint32_t step = 1u << kLogNMax;
    for (uint32_t q = kSmallPrimeMax / step;; --q) {
      const uint64_t p = (uint64_t)q * step + 1;
      if (p <= (1ull << 30)) break;
      if (p <= kSmallPrimeMax && is_prime_u32((uint32_t)p)) H.p.push_back((uint32_t)p);
    }
    H.n_small = (int)H.p.size();
    for (uint32_t q = ((1u << 31) - 2) / step;; --q) {
      const uint64_t p = (uint64_t)q * step + 1;
      if (p <= kSmallPrimeMax) break;
      if (p < (1ull << 31) && is_prime_u32((uint32_t)p)) H.p.push_back((uint32_t)p);
    }
    const int T = (int)H.p.size();
    H.pc.resize(T);
    H.pw.resize((size_t)T * (kMaxLimbs + 1));
    H.mpw.resize((size_t)T * (kMaxLimbs + 1));
    H.lg_prefix.resize(T + 1);
    H.lg_prefix[0] = 0;
    for (int i = 0; i < T; ++i) {
      const uint32_t p = H.p[i];
      PrimeConst c;
      c.p = p;
      c.pinv = host_pinv(p);
      c.one_m = (uint32_t)((1ull << 32) % p);
      c.r2 = (uint32_t)(((uint64_t)c.one_m << 32) % p);
      c.g = primitive_root(p);
      c.c_m = host_to_mont(coset_rep(p, c.g), p);
      c.half = (p - 1) / 2;
      c.pad = 0;
      H.pc[i] = c;
      // pw[l] = 2^(32 l + 64) mod p, mpw[l] = 2^(32 l + 32) mod p
      uint64_t m = c.one_m;  // 2^32
      for (int l = 0; l <= kMaxLimbs; ++l) {
        H.mpw[(size_t)i * (kMaxLimbs + 1) + l] = (uint32_t)m;
        H.pw[(size_t)i * (kMaxLimbs + 1) + l] = (uint32_t)((m << 32) % p);
        m = (m << 32) % p;
      }
      H.lg_prefix[i + 1] = H.lg_prefix[i] + log2_q16_down_u31(p);
    }
  });
  return H;
}

// ------------------------------------------------------------------------------------
// device tables
// ------------------------------------------------------------------------------------
__global__ void k_init_transform(const PrimeConst* pc, const uint32_t* omega_m,
                                 const uint32_t* ginv_m, int Tt, int NT, int logNT,
                                 uint32_t* tw, uint32_t* itw, uint32_t* cp, uint32_t* icp,
                                 uint32_t* ninv) {
  const int64_t total = (int64_t)Tt * NT;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / NT);
    const int i = (int)(idx - (int64_t)q * NT);
    const PrimeConst c = pc[q];
    const Mod M{c.p, c.pinv};
    if (i < NT / 2) {
      const uint32_t w = omega_m[q];
      const uint32_t wi = mpow(w, (uint32_t)i, c.one_m, M);
      tw[(int64_t)q * (NT / 2) + i] = wi;
      // omega^-i = omega^(NT - i)
      itw[(int64_t)q * (NT / 2) + i] = i ? mpow(w, (uint32_t)(NT - i), c.one_m, M) : c.one_m;
    }
    cp[idx] = mpow(c.c_m, (uint32_t)i, c.one_m, M);
    // standard form of c^-i: REDC of its Montgomery form
    icp[idx] = redc((uint64_t)mpow(ginv_m[q], (uint32_t)i, c.one_m, M), c.p, c.pinv);
    if (i <= kLogNMax) {
      // 2^-i in Montgomery form: (2^-1)^i with 2^-1 = (p + 1) / 2
      const uint32_t half_m = redc((uint64_t)((c.p + 1) / 2) * c.r2, c.p, c.pinv);
      ninv[q * (kLogNMax + 1) + i] = mpow(half_m, (uint32_t)i, c.one_m, M);
    }
  }
}

// packed twiddles: P[len + j] = omega_{2 len}^{+-j} = tw[j NT / (2 len)] for len = 1 .. NT/2,
// j < len (entry 0 holds 1); every transform stage then reads consecutive entries
__global__ void k_init_packed(const PrimeConst* pc, int Tt, int NT, int logNT, const uint32_t* tw,
                              const uint32_t* itw, uint32_t* twp, uint32_t* itwp) {
  const int64_t total = (int64_t)Tt * NT;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / NT);
    const int t = (int)(idx - (int64_t)q * NT);
    if (t == 0) {
      twp[idx] = pc[q].one_m;
      itwp[idx] = pc[q].one_m;
      continue;
    }
    const int lg = 31 - __clz(t);
    const int64_t src = (int64_t)q * (NT / 2) + ((int64_t)(t - (1 << lg)) << (logNT - lg - 1));
    twp[idx] = tw[src];
    itwp[idx] = itw[src];
  }
}

// the Shoup pairs of the first 32 packed twiddles of every prime
__global__ void k_init_shoup(const PrimeConst* pc, int Tt, int NT, const uint32_t* twp, uint32_t* tws) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < Tt * 32; idx += gridDim.x * blockDim.x) {
    const int q = idx >> 5, j = idx & 31;
    const uint32_t p = pc[q].p;
    // j = 0 holds the pair of 1 (the factor of the lanes that only add in a shuffle stage)
    const uint32_t w = j ? redc((uint64_t)twp[(int64_t)q * NT + j], p, pc[q].pinv) : 1u;
    tws[2 * idx] = w;
    tws[2 * idx + 1] = (uint32_t)(((uint64_t)w << 32) / p);
  }
}

__global__ void k_init_garner(const PrimeConst* pc, int Tg, uint32_t* ginv) {
  const int64_t total = (int64_t)Tg * Tg;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / Tg);
    const int b = (int)(idx - (int64_t)a * Tg);
    if (a == b) {
      ginv[idx] = 0;
      continue;
    }
    const PrimeConst cb = pc[b];
    const Mod M{cb.p, cb.pinv};
    const uint32_t pa = pc[a].p % cb.p;
    const uint32_t pa_m = redc((uint64_t)pa * cb.r2, cb.p, cb.pinv);
    ginv[idx] = minv(pa_m, cb.one_m, M);
  }
}

// prefix products P_j = p_0 ... p_{j-1} of the first Tg table primes, one warp: every
// step multiplies the previous row by p_j, lanes own 32-limb chunks, carries between
// lanes are resolved with generate/propagate ballots
__global__ void k_init_prefix(const PrimeConst* pc, int Tg, int LPP, uint32_t* pp) {
  const int lane = threadIdx.x & 31;
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  for (int l = lane; l < LPP; l += 32) pp[l] = (l == 0) ? 1u : 0u;
  __syncwarp();
  int len = 1;  // limbs in use
  for (int j = 0; j < Tg; ++j) {
    const uint32_t p = pc[j].p;
    const uint32_t* src = pp + (size_t)j * LPP;
    uint32_t* dst = pp + (size_t)(j + 1) * LPP;
    const int nlen = len + 1 < LPP ? len + 1 : LPP;
    uint32_t cin = 0, hprev = 0;
    for (int b = 0; b < LPP; b += 32) {
      const int l = b + lane;
      const uint32_t v = (l < len) ? src[l] : 0u;
      const uint64_t prod = (uint64_t)v * p;
      const uint32_t lo = (uint32_t)prod, hi = (uint32_t)(prod >> 32);
      uint32_t hin = __shfl_up_sync(0xffffffffu, hi, 1);
      if (lane == 0) hin = hprev;
      const uint32_t s = lo + hin;
      const uint32_t G = __ballot_sync(0xffffffffu, s < lo);
      const uint32_t Pm = __ballot_sync(0xffffffffu, s == 0xffffffffu) & ~G;
      const uint32_t X = G | Pm;
      const uint64_t S = (uint64_t)X + G + cin;
      const uint32_t C = (uint32_t)S ^ X ^ G;
      if (l < LPP) dst[l] = (l < nlen) ? s + ((C >> lane) & 1u) : 0u;
      cin = (uint32_t)(S >> 32);
      hprev = __shfl_sync(0xffffffffu, hi, 31);
    }
    len = nlen;
    __syncwarp();
  }
}

// weighted-sum tables: block k - 1 handles k primes, its threads take i < k:
// M_k[i] = P_k / p_i by exact long division of the prefix product P_k (row k of pp) by p_i,
// and y_k[i] = (prod_{j<k, j!=i} p_j)^-1 mod p_i in Montgomery form
__global__ void k_init_ws(const PrimeConst* pc, const uint32_t* pp, int LPP, int WK,
                          const int64_t* moff, const int32_t* yoff, uint32_t* wsm, uint32_t* wsy) {
  for (int k = blockIdx.x + 1; k <= WK; k += gridDim.x) {
    const int L = ws_len(k);
    const uint32_t* Pk = pp + (size_t)k * LPP;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const uint32_t p = pc[i].p;
      uint32_t* dst = wsm + moff[k] + (int64_t)i * L;
      uint64_t rem = 0;
      for (int l = L - 1; l >= 0; --l) {
        const uint64_t cur = (rem << 32) | (l < LPP ? Pk[l] : 0u);
        dst[l] = (uint32_t)(cur / p);
        rem = cur % p;
      }
      const Mod M{p, pc[i].pinv};
      uint32_t prod = pc[i].one_m;
      for (int j = 0; j < k; ++j) {
        if (j == i) continue;
        const uint32_t pj = pc[j].p % p;
        prod = mmul(prod, redc((uint64_t)pj * pc[i].r2, p, pc[i].pinv), M);
      }
      wsy[yoff[k] + i] = minv(prod, pc[i].one_m, M);
    }
  }
}

static int cu_fail(cudaError_t e) { return e == cudaSuccess ? 0 : kErrCuda; }

int DeviceTables::init(cudaStream_t s) {
  const HostPrimes& H = host_primes();
  T = (int)H.p.size();
  if (cudaMalloc(&pc, sizeof(PrimeConst) * T) != cudaSuccess) return kErrCuda;
  if (cudaMalloc(&pw, sizeof(uint32_t) * H.pw.size()) != cudaSuccess) return kErrCuda;
  if (cudaMalloc(&mpw, sizeof(uint32_t) * H.mpw.size()) != cudaSuccess) return kErrCuda;
  if (cudaMalloc(&lgp, sizeof(int64_t) * H.lg_prefix.size()) != cudaSuccess) return kErrCuda;
  int rc = 0;
  rc |= cu_fail(cudaMemcpyAsync(pc, H.pc.data(), sizeof(PrimeConst) * T, cudaMemcpyHostToDevice, s));
  rc |= cu_fail(cudaMemcpyAsync(pw, H.pw.data(), sizeof(uint32_t) * H.pw.size(), cudaMemcpyHostToDevice, s));
  rc |= cu_fail(cudaMemcpyAsync(mpw, H.mpw.data(), sizeof(uint32_t) * H.mpw.size(), cudaMemcpyHostToDevice, s));
  rc |= cu_fail(cudaMemcpyAsync(lgp, H.lg_prefix.data(), sizeof(int64_t) * H.lg_prefix.size(),
                                cudaMemcpyHostToDevice, s));
  if (rc) return kErrCuda;
  return cu_fail(cudaStreamSynchronize(s));
}

void DeviceTables::release() {
  for (void* p : {(void*)pc, (void*)pw, (void*)mpw, (void*)lgp, (void*)tw, (void*)itw,
                  (void*)cp, (void*)icp, (void*)ninv, (void*)ginv, (void*)pp, (void*)ws_m,
                  (void*)ws_y, (void*)ws_moff, (void*)ws_yoff, (void*)q62, (void*)twp, (void*)itwp,
                  (void*)tws})
    if (p) cudaFree(p);
  twp = itwp = tws = nullptr;
  ws_m = ws_y = q62 = nullptr;
  ws_moff = nullptr;
  ws_yoff = nullptr;
  WK = 0;
  pp = nullptr;
  LPP = 0;
  pc = nullptr;
  pw = mpw = tw = itw = cp = icp = ninv = ginv = nullptr;
  lgp = nullptr;
  Tt = NT = logNT = Tg = 0;
}

int DeviceTables::ensure(int needT, int needLogN, cudaStream_t s) {
  if (needT > T || needLogN > kLogNMax) return kErrRange;
  if (needT <= Tt && needLogN <= logNT && needT <= Tg) return 0;
  const HostPrimes& H = host_primes();
  int newT = Tt;
  if (needT > newT) {
    newT = needT + needT / 2 + 32;
    if (newT > T) newT = T;
  }
  int newLog = needLogN > logNT ? needLogN : logNT;
  if (newLog < 6) newLog = 6;
  const int newNT = 1 << newLog;
  // finish any work that may still read the old tables
  if (cudaStreamSynchronize(s) != cudaSuccess) return kErrCuda;
  uint32_t *ntw = nullptr, *nitw = nullptr, *ncp = nullptr, *nicp = nullptr, *nninv = nullptr,
           *nginv = nullptr, *omega = nullptr, *gi = nullptr, *ntwp = nullptr, *nitwp = nullptr,
           *ntws = nullptr;
  int rc = 0;
  rc |= cu_fail(cudaMalloc(&ntw, sizeof(uint32_t) * (size_t)newT * (newNT / 2)));
  rc |= cu_fail(cudaMalloc(&nitw, sizeof(uint32_t) * (size_t)newT * (newNT / 2)));
  rc |= cu_fail(cudaMalloc(&ntwp, sizeof(uint32_t) * (size_t)newT * newNT));
  rc |= cu_fail(cudaMalloc(&nitwp, sizeof(uint32_t) * (size_t)newT * newNT));
  rc |= cu_fail(cudaMalloc(&ntws, sizeof(uint32_t) * (size_t)newT * 64));
  rc |= cu_fail(cudaMalloc(&ncp, sizeof(uint32_t) * (size_t)newT * newNT));
  rc |= cu_fail(cudaMalloc(&nicp, sizeof(uint32_t) * (size_t)newT * newNT));
  rc |= cu_fail(cudaMalloc(&nninv, sizeof(uint32_t) * (size_t)newT * (kLogNMax + 1)));
  rc |= cu_fail(cudaMalloc(&nginv, sizeof(uint32_t) * (size_t)newT * newT));
  rc |= cu_fail(cudaMalloc(&omega, sizeof(uint32_t) * newT));
  const int newLPP = (31 * newT + 31) / 32 + 2;
  uint32_t* npp = nullptr;
  rc |= cu_fail(cudaMalloc(&npp, sizeof(uint32_t) * (size_t)(newT + 1) * newLPP));
  rc |= cu_fail(cudaMalloc(&gi, sizeof(uint32_t) * newT));
  if (rc) {
    for (void* p : {(void*)ntw, (void*)nitw, (void*)ncp, (void*)nicp, (void*)nninv, (void*)nginv,
                    (void*)omega, (void*)gi, (void*)ntwp, (void*)nitwp, (void*)ntws})
      if (p) cudaFree(p);
    return kErrNoMem;
  }
  std::vector<uint32_t> om(newT), gim(newT);
  for (int q = 0; q < newT; ++q) {
    const uint32_t p = H.p[q];
    const uint32_t g = H.pc[q].g;
    const uint32_t cr = redc((uint64_t)H.pc[q].c_m, p, H.pc[q].pinv);  // c in standard form
    om[q] = host_to_mont(host_powmod(g, (p - 1) / newNT, p), p);
    gim[q] = host_to_mont(host_powmod(cr, p - 2, p), p);
  }
  rc |= cu_fail(cudaMemcpyAsync(omega, om.data(), sizeof(uint32_t) * newT, cudaMemcpyHostToDevice, s));
  rc |= cu_fail(cudaMemcpyAsync(gi, gim.data(), sizeof(uint32_t) * newT, cudaMemcpyHostToDevice, s));
  k_init_transform<<<1024, 256, 0, s>>>(pc, omega, gi, newT, newNT, newLog, ntw, nitw, ncp, nicp, nninv);
  rc |= cu_fail(cudaGetLastError());
  k_init_packed<<<1024, 256, 0, s>>>(pc, newT, newNT, newLog, ntw, nitw, ntwp, nitwp);
  rc |= cu_fail(cudaGetLastError());
  k_init_shoup<<<(newT * 32 + 255) / 256, 256, 0, s>>>(pc, newT, newNT, ntwp, ntws);
  rc |= cu_fail(cudaGetLastError());
  k_init_garner<<<1024, 256, 0, s>>>(pc, newT, nginv);
  rc |= cu_fail(cudaGetLastError());
  k_init_prefix<<<1, 32, 0, s>>>(pc, newT, newLPP, npp);
  rc |= cu_fail(cudaGetLastError());
  // weighted-sum reconstruction tables for k <= newWK
  const int newWK = newT < kWsMaxK ? newT : kWsMaxK;
  std::vector<int64_t> moff(newWK + 2, 0);
  std::vector<int32_t> yoff(newWK + 2, 0);
  for (int kk = 1; kk <= newWK; ++kk) {
    moff[kk + 1] = moff[kk] + (int64_t)kk * ws_len(kk);
    yoff[kk + 1] = yoff[kk] + kk;
  }
  uint32_t *nwsm = nullptr, *nwsy = nullptr, *nq62 = nullptr;
  int64_t* nmoff = nullptr;
  int32_t* nyoff = nullptr;
  rc |= cu_fail(cudaMalloc(&nwsm, sizeof(uint32_t) * std::max<int64_t>(moff[newWK + 1], 1)));
  rc |= cu_fail(cudaMalloc(&nwsy, sizeof(uint32_t) * std::max(yoff[newWK + 1], 1)));
  rc |= cu_fail(cudaMalloc(&nmoff, sizeof(int64_t) * (newWK + 2)));
  rc |= cu_fail(cudaMalloc(&nyoff, sizeof(int32_t) * (newWK + 2)));
  rc |= cu_fail(cudaMalloc(&nq62, sizeof(uint32_t) * newT));
  if (!rc) {
    std::vector<uint32_t> q(newT);
    for (int i = 0; i < newT; ++i) q[i] = (uint32_t)((1ull << 62) / H.p[i]);
    rc |= cu_fail(cudaMemcpyAsync(nmoff, moff.data(), sizeof(int64_t) * (newWK + 2), cudaMemcpyHostToDevice, s));
    rc |= cu_fail(cudaMemcpyAsync(nyoff, yoff.data(), sizeof(int32_t) * (newWK + 2), cudaMemcpyHostToDevice, s));
    rc |= cu_fail(cudaMemcpyAsync(nq62, q.data(), sizeof(uint32_t) * newT, cudaMemcpyHostToDevice, s));
    rc |= cu_fail(cudaStreamSynchronize(s));  // the host vectors go out of scope
    k_init_ws<<<newWK > 0 ? newWK : 1, 128, 0, s>>>(pc, npp, newLPP, newWK, nmoff, nyoff, nwsm, nwsy);
    rc |= cu_fail(cudaGetLastError());
  }
  rc |= cu_fail(cudaStreamSynchronize(s));
  cudaFree(omega);
  cudaFree(gi);
  for (void* p : {(void*)tw, (void*)itw, (void*)cp, (void*)icp, (void*)ninv, (void*)ginv, (void*)pp,
                  (void*)ws_m, (void*)ws_y, (void*)ws_moff, (void*)ws_yoff, (void*)q62, (void*)twp,
                  (void*)itwp, (void*)tws})
    if (p) cudaFree(p);
  twp = ntwp;
  itwp = nitwp;
  tws = ntws;
  ws_m = nwsm;
  ws_y = nwsy;
  ws_moff = nmoff;
  ws_yoff = nyoff;
  q62 = nq62;
  WK = newWK;
  ws_m_words = std::max<int64_t>(moff[newWK + 1], 1);
  pp = npp;
  LPP = newLPP;
  tw = ntw;
  itw = nitw;
  cp = ncp;
  icp = nicp;
  ninv = nninv;
  ginv = nginv;
  Tt = Tg = newT;
  NT = newNT;
  logNT = newLog;
  ++generation;
  return rc ? kErrCuda : 0;
}

Tables DeviceTables::view() const {
  Tables t;
  t.pc = pc;
  t.pw = pw;
  t.mpw = mpw;
  t.lg_prefix = lgp;
  t.tw = tw;
  t.itw = itw;
  t.twp = twp;
  t.itwp = itwp;
  t.tws = tws;
  t.cp = cp;
  t.icp = icp;
  t.ninv = ninv;
  t.ginv = ginv;
  t.pp = pp;
  t.LPP = LPP;
  t.ws_m = ws_m;
  t.ws_moff = ws_moff;
  t.ws_y = ws_y;
  t.ws_yoff = ws_yoff;
  t.q62 = q62;
  t.ws_m_words = ws_m_words;
  t.WK = WK;
  t.T = T;
  t.Tt = Tt;
  t.NT = NT;
  t.logNT = logNT;
  t.Tg = Tg;
  return t;
}

}  // namespace bs
