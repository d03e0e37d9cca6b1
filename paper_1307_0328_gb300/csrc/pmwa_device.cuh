// pmwa_device.cuh -- device building blocks of the PMWA sweep: counter-based
// random numbers, deterministic exponentials, the worm-number sampler of
// Eq. 1, lattice geometry and the per-site event slots.
//
// Every floating-point operation that decides an integer (ziggurat wedge
// test, grid gaps, boundary heat-bath) uses explicit round-to-nearest
// intrinsics, so no multiply-add is ever contracted and the result is the
// IEEE binary64 result of the written expression.
#pragma once
#include <cstdint>

#include "pmwa_internal.h"

namespace pmwa {

__constant__ double c_zX[257];
__constant__ double c_zF[257];
__constant__ double c_zW[256];
__constant__ double c_zS[256];
__constant__ unsigned long long c_zK[256];
__constant__ unsigned long long c_zXF[256];
__constant__ unsigned long long c_zRF;
__constant__ double c_zR;
// Taylor coefficients 1/n!, n = 0..24: the correctly rounded quotients
// 1.0 / n! of exact factorials, computed on the host.
__constant__ double c_inv_fact[25];

// Every translation unit that includes this header owns its own copy of the
// constant tables above (no relocatable device code), so each unit uploads
// them through this function.
static int upload_constants(const Zig& z) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_zX, z.X, sizeof z.X))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zF, z.F, sizeof z.F))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zW, z.W, sizeof z.W))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zS, z.S, sizeof z.S))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zK, z.K, sizeof z.K))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zR, &z.R, sizeof z.R))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zXF, z.XF, sizeof z.XF))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zRF, &z.RF, sizeof z.RF))) return int(e);
  double inv_fact[25];
  double fact = 1.0;
  for (int n = 0; n <= 24; ++n) {
    if (n > 0) fact = fact * double(n);  // the same rounded running products as
    inv_fact[n] = 1.0 / fact;            // the CPU reference computes
  }
  if ((e = cudaMemcpyToSymbol(c_inv_fact, inv_fact, sizeof inv_fact))) return int(e);
  return 0;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products
// mixed into the other two words, key advanced by the Weyl increments.
struct P4 { uint32_t x, y, z, w; };

__device__ __forceinline__ P4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return P4{c0, c1, c2, c3};
}

// Sequence of 64-bit words of the blocks with counter (block, unit, c2, sweep):
// word w is the low (w even) or high (w odd) half of block w/2.
struct Stream {
  uint32_t k0, k1, unit, c2, sweep;
  uint64_t pos;
  P4 blk;
  uint64_t cached;  // block index held in blk, or ~0
  __device__ void init(uint32_t key0, uint32_t key1, uint32_t u, uint32_t cc2, uint32_t sw) {
    k0 = key0; k1 = key1; unit = u; c2 = cc2; sweep = sw; pos = 0; cached = ~0ull;
  }
  __device__ uint64_t word() {
    const uint64_t b = pos >> 1;
    if (b != cached) { blk = philox(uint32_t(b), unit, c2, sweep, k0, k1); cached = b; }
    const uint64_t w = (pos & 1) ? (uint64_t(blk.z) | (uint64_t(blk.w) << 32))
                                 : (uint64_t(blk.x) | (uint64_t(blk.y) << 32));
    ++pos;
    return w;
  }
};

// The same word sequence for a warp that runs one scalar chain (every lane
// calls word() with the same state, all lanes active): lane j holds block
// base + j of a 32-block window and each word is fetched by two shuffles,
// so the warp evaluates Philox once per 64 words instead of once per 2.
struct WarpStream {
  uint32_t k0, k1, unit, c2, sweep;
  uint64_t pos;
  uint64_t base;  // first block of the window the lanes hold
  P4 mine;        // block base + lane
  __device__ void init(uint32_t key0, uint32_t key1, uint32_t u, uint32_t cc2, uint32_t sw) {
    k0 = key0; k1 = key1; unit = u; c2 = cc2; sweep = sw; pos = 0;
    base = ~0ull - 63;  // (b - base = b + 64 >= 32: the first word fills the window)
  }
  __device__ uint64_t word() {
    const uint64_t b = pos >> 1;
    if (b - base >= 32) {
      base = b & ~31ull;
      mine = philox(uint32_t(base) + (threadIdx.x & 31), unit, c2, sweep, k0, k1);
    }
    const int src = int(b - base);
    const bool odd = pos & 1;
    const uint32_t lo = __shfl_sync(0xffffffffu, odd ? mine.z : mine.x, src);
    const uint32_t hi = __shfl_sync(0xffffffffu, odd ? mine.w : mine.y, src);
    ++pos;
    return uint64_t(lo) | (uint64_t(hi) << 32);
  }
};

__device__ __forceinline__ uint32_t c2_word(uint32_t phase, uint32_t pass, uint32_t replica) {
  return phase | (pass << 4) | (replica << 16);
}

// ---------------------------------------------------------------------------
// Deterministic e^x: x = k ln2 + r with ln2 = LN2_HI (24 significant bits) +
// LN2_LO, then the Taylor polynomial of e^r to degree 13 (Horner), then the
// exact power of two.  Coefficients 1/n! are the correctly rounded quotients
// of exact factorials.
__device__ __forceinline__ double pow2i(int k) {
  return __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ inline double exp_det(double x) {
  if (x != x) return x;
  if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
  if (x < -745.0) return 0.0;
  const double kd = floor(__dadd_rn(__dmul_rn(x, 1.4426950408889634), 0.5));
  const int k = int(kd);
  const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kd, 0.693147182464599609375)),
                             __dmul_rn(kd, -1.9046542999577678e-09));
  double p = c_inv_fact[13];
#pragma unroll
  for (int n = 12; n >= 0; --n) p = __dadd_rn(__dmul_rn(p, r), c_inv_fact[n]);
  if (k >= -1022) return __dmul_rn(p, pow2i(k));
  return __dmul_rn(__dmul_rn(p, pow2i(k + 600)), pow2i(-600));
}

// e^x - 1 on [-1, 1]: the Taylor polynomial (no constant term) of degree
// 7, 9, 13 or 19 as |x| <= 2^-6, 2^-4, 2^-2 or 1 (truncation below 2^-57
// relative), Horner's rule with explicit rounding; exp_det(x) - 1 beyond.
__device__ inline double expm1_det(double x) {
  if (!(x <= 1.0 && x >= -1.0)) return __dsub_rn(exp_det(x), 1.0);
  const double ax = fabs(x);
  const int d = (ax <= 0x1p-6) ? 7 : (ax <= 0x1p-4) ? 9 : (ax <= 0x1p-2) ? 13 : 19;
  double p = c_inv_fact[d];
  for (int n = d - 1; n >= 1; --n) p = __dadd_rn(__dmul_rn(p, x), c_inv_fact[n]);
  return __dmul_rn(p, x);
}

// x tanh x / x coth x building blocks (x >= 0): with e = e^{-2x} - 1,
// tanh x = -e / (2 + e) and coth x = (2 + e) / -e.
__device__ inline double g_sigma(int sigma, double x) {
  const double e = expm1_det(__dmul_rn(-2.0, x));
  return sigma ? __ddiv_rn(__dadd_rn(2.0, e), -e) : __ddiv_rn(-e, __dadd_rn(2.0, e));
}

// x g_sigma(x) for the worm-density estimator (an FP64 observable, not a
// decision): the power series in y = x^2, x tanh x = sum_n a_n y^n and
// x coth x = sum_n b_n y^n with a_n = 2^{2n} (2^{2n} - 1) B_{2n} / (2n)! and
// b_n = 2^{2n} B_{2n} / (2n)! (B the Bernoulli numbers); 6 terms for
// y <= 1/400 and 16 for y <= 1/4 keep the truncation below 1e-17, larger x
// go through expm1_det.
__constant__ double c_xtanh[16] = {1.0, -0.3333333333333333, 0.13333333333333333, -0.05396825396825397, 0.021869488536155203, -0.008863235529902197, 0.003592128036572481, -0.0014558343870513183, 0.000590027440945586, -0.00023912911424355248, 9.691537956929451e-05, -3.927832388331683e-05, 1.5918905069328964e-05, -6.451689215655431e-06, 2.6147711512907546e-06, -1.0597268320104654e-06};
__constant__ double c_xcoth[17] = {1.0, 0.3333333333333333, -0.022222222222222223, 0.0021164021164021165, -0.00021164021164021165, 2.1377799155576935e-05, -2.1644042808063972e-06, 2.1925947851873778e-07, -2.2214608789979678e-08, 2.2507846516808994e-09, -2.2805151204592183e-10, 2.3106432599002624e-11, -2.3411706819824882e-12, 2.3721017400233653e-13, -2.4034415333307705e-14, 2.4351954029183367e-15, -2.4673688045172075e-16};

__device__ inline double xg_sigma(int sigma, double x) {
  const double y = x * x;
  int n;
  if (y <= 2.5e-3) n = 6;
  else if (y <= 0.25) n = 16;
  else return __dmul_rn(x, g_sigma(sigma, x));
  double p;
  if (sigma) {
    p = c_xcoth[n - 1];
    for (int k = n - 2; k >= 0; --k) p = fma(p, y, c_xcoth[k]);
    return p;
  }
  p = c_xtanh[n - 1];
  for (int k = n - 2; k >= 0; --k) p = fma(p, y, c_xtanh[k]);
  return p * y;
}

// The same two series in fixed point, for the per-interval terms of the
// estimator: coefficients a_n 2^62 and b_n 2^62 rounded to nearest (exact
// rationals from the Bernoulli numbers), Horner's rule on signed 64-bit
// words with y 2^64 = (x 2^64)^2 / 2^64.  The terms kept (5, 8 or 19 for
// tanh and 5, 7 or 13 for coth as x < 2^-5, 2^-3, 2^-1) leave a truncation
// below 2^-63; each product is floored, so a term is within (n + 1) 2^-62
// of x g_sigma(x).  No floating point is used, so the sum of the terms of a
// site is exact and independent of the order of summation.
__constant__ long long c_xtanh_fx[19] = {
    4611686018427387904ll, -1537228672809129301ll, 614891469123651721ll, -248884642264335220ll,
    100855214512344991ll, -40874459371278820ll, 16565766642662335ll, -6713851087910371ll,
    2721021299897250ll, -1102788392755917ll, 446943300930299ll, -181139297079955ll,
    73412991936897ll, -29753164951077ll, 12058503559795ll, -4887127414535ll,
    1980678137006ll, -802738613024ll, 325337705708ll};
__constant__ long long c_xcoth_fx[13] = {
    4611686018427387904ll, 1537228672809129301ll, -102481911520608620ll, 9760182049581773ll,
    -976018204958177ll, 98587697470523ll, -9981552960019ll, 1011155871493ll,
    -102446800762ll, 10379912109ll, -1051701970ll, 106559612ll, -10796744ll};

// x g_sigma(x) 2^62 for x = I beta eta / 2^59 (XQ: beta eta 2^5 as a grid
// scale, so that x 2^64 = (I m) >> sh); false when x >= 1/2, where the
// caller uses the binary64 form.
__device__ __forceinline__ bool xg_fix(int sigma, uint64_t I, GridScale XQ, uint64_t& out) {
  const uint64_t hi = __umul64hi(I, XQ.m), lo = I * XQ.m;
  uint64_t X;
  if (XQ.sh >= 64) {
    X = hi >> (XQ.sh - 64);
  } else {
    if (hi >> XQ.sh) return false;
    X = (hi << (64 - XQ.sh)) | (lo >> XQ.sh);
  }
  if (X >= (1ull << 63)) return false;
  const long long Y = (long long)__umul64hi(X, X);
  const int band = (X < (1ull << 59)) ? 0 : (X < (1ull << 61)) ? 1 : 2;
  long long p;
  if (sigma) {
    const int n = band == 0 ? 5 : band == 1 ? 7 : 13;
    p = c_xcoth_fx[n - 1];
    for (int k = n - 2; k >= 0; --k) p = c_xcoth_fx[k] + __mul64hi(p, Y);
    out = uint64_t(p);
  } else {
    const int n = band == 0 ? 5 : band == 1 ? 8 : 19;
    p = c_xtanh_fx[n - 1];
    for (int k = n - 2; k >= 0; --k) p = c_xtanh_fx[k] + __mul64hi(p, Y);
    out = uint64_t(__mul64hi(p, Y));
  }
  return true;
}

// ---------------------------------------------------------------------------
// Ziggurat tables as seen by a kernel: the two tables of the fast path (the
// inner-rectangle thresholds K and the fixed-point strip edges XF) copied
// into shared memory, because the strip index differs from lane to lane
// (constant memory would serialise); the wedge test (about 1 % of the words)
// reads W and F from constant memory.
struct ZigTab {
  const unsigned long long* K;   // [256] inner-rectangle threshold
  const unsigned long long* XF;  // [256] X[i] 2^58
  int zcap;                      // words per deviate (64; Dev::zig_cap)
  int wtries;                    // proposals of the Eq. 1 sampler (128; Dev::worm_tries)
};
constexpr int kZigBytes = 256 * 8 + 256 * 8;

// copy the tables into `buf` (kZigBytes, 8-byte aligned); all threads
// participate; the caller synchronises before use
__device__ inline ZigTab zig_stage(unsigned char* buf, int zcap = 64, int wtries = 128) {
  unsigned long long* K = reinterpret_cast<unsigned long long*>(buf);
  unsigned long long* XF = reinterpret_cast<unsigned long long*>(buf + 256 * 8);
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    K[i] = c_zK[i];
    XF[i] = c_zXF[i];
  }
  return ZigTab{K, XF, zcap, wtries};
}

__device__ __forceinline__ uint64_t zfix_add(uint64_t a, uint64_t b) { return (a > ~0ull - b) ? ~0ull : a + b; }

// Unit exponential E from the ziggurat of Marsaglia and Tsang (2000), in
// fixed point E 2^58: strip i from the low 8 bits of a word, a 53-bit
// uniform u from its high bits, the point x = u X[i] / 2^53 as the exact
// product (u XF[i]) >> 53; accept when u < K[i]; strip 0 past R restarts at
// R + new deviate; else a binary64 wedge test y < e^-x with a second word.
// <= z.zcap (64) words.
template <class St>
__device__ inline uint64_t zig_exp(const ZigTab& z, St& s, int* bad) {
  uint64_t acc = 0;
  for (int tries = 0; tries < z.zcap; ++tries) {
    const uint64_t w = s.word();
    const unsigned i = unsigned(w & 255u);
    const uint64_t u = w >> 11;
    const uint64_t xf0 = z.XF[i];
    const uint64_t xf = (__umul64hi(u, xf0) << 11) | ((u * xf0) >> 53);
    if (u < z.K[i]) return zfix_add(acc, xf);
    if (i == 0) { acc = zfix_add(acc, c_zRF); continue; }
    const double x = __dmul_rn(__ull2double_rn(u), c_zW[i]);
    const uint64_t w2 = s.word();
    const double t1 = __dmul_rn(__ull2double_rn(w2 >> 11), 0x1p-53);
    const double t2 = __dsub_rn(c_zF[i + 1], c_zF[i]);
    const double y = __dadd_rn(c_zF[i], __dmul_rn(t1, t2));
    // The test y < exp_det(-x), decided first by bounds of e^-x on the
    // strip's wedge [a, b] = [X[i+1], X[i]]: the tangent at a below
    // (e^-x >= e^-a (1 - (x - a))) and the chord above (e^-x is convex).
    // Away from the curve by more than eps = F[i+1] 2^-40 -- far beyond the
    // rounding of the bounds, of the tables and of exp_det (a few units in
    // the last place) -- the bounds give the same answer as the exact test,
    // which runs only inside that margin.
    const double fa = c_zF[i + 1], dl = __dsub_rn(x, c_zX[i + 1]), eps = __dmul_rn(fa, 0x1p-40);
    if (y < __dsub_rn(__dmul_rn(fa, __dsub_rn(1.0, dl)), eps)) return zfix_add(acc, xf);
    if (y > __dadd_rn(__dadd_rn(fa, __dmul_rn(dl, c_zS[i])), eps)) continue;
    if (y < exp_det(-x)) return zfix_add(acc, xf);
  }
  *bad = PMWA_ETIMEOUT;
  return 0;
}

// Gap of a Bernoulli process of mean spacing S on an integer grid:
// 1 + floor(E S) from the exact 128-bit product (E 2^58) m, shifted right
// by sh (22 <= sh <= 82); saturates at 2^62.
__device__ __forceinline__ uint64_t grid_gap(uint64_t Ef, GridScale S) {
  const uint64_t hi = __umul64hi(Ef, S.m), lo = Ef * S.m;
  uint64_t g;
  if (S.sh >= 64) {
    g = hi >> (S.sh - 64);
  } else {
    if (hi >> S.sh) return kTwo62;
    g = (hi << (64 - S.sh)) | (lo >> S.sh);
  }
  if (g >= kTwo62) return kTwo62;
  return 1 + g;
}

// Eq. 1 for hard-core bosons: worms on an interval of M worm grid points with
// parity sigma.  Rate-eta Bernoulli/Poisson process (mean spacing SW grid
// points) conditioned on the parity of its count; for sigma = 1 and x <= 1
// (M <= SWI) the proposal is 1 + count, kept with probability 1/n when n is
// odd, the extra worm uniform on the interval (a clash rejects).  Returns the
// count (offsets sorted in offs[0..n)), or -1 with *bad set.
template <int MAXN, class St>
__device__ int sample_worms(const ZigTab& z, St& s, uint64_t M, int sigma, GridScale SW, uint64_t SWI,
                            uint64_t* offs, int* bad) {
  if (M == 0) { if (sigma) { *bad = PMWA_EINVARIANT; return -1; } return 0; }
  for (int tries = 0; tries < z.wtries; ++tries) {
    int n = 0;
    bool first = true;
    uint64_t pos = 0;
    for (;;) {
      const uint64_t E = zig_exp(z, s, bad);
      const uint64_t g = grid_gap(E, SW);
      const uint64_t nxt = first ? g - 1 : pos + g;
      first = false;
      if (nxt >= M) break;
      pos = nxt;
      if (n >= MAXN) { *bad = PMWA_ECAPACITY; return -1; }
      offs[n++] = pos;
    }
    if (sigma == 1 && M <= SWI) {
      const int ntot = n + 1;
      if ((ntot & 1) == 0) continue;
      if (__umul64hi(s.word(), uint64_t(ntot)) != 0) continue;
      const uint64_t extra = __umul64hi(s.word(), M);
      int at = n;
      bool clash = false;
      for (int k = 0; k < n; ++k) {
        if (offs[k] == extra) { clash = true; break; }
        if (offs[k] > extra) { at = k; break; }
      }
      if (clash) continue;
      if (n >= MAXN) { *bad = PMWA_ECAPACITY; return -1; }
      for (int k = n; k > at; --k) offs[k] = offs[k - 1];
      offs[at] = extra;
      return ntot;
    }
    if ((n & 1) == sigma) return n;
  }
  *bad = PMWA_ETIMEOUT;
  return -1;
}

// An instance whose error word is set has an undefined configuration:
// every kernel that reads it leaves at once.  All threads of the CTA call
// this together (it is a barrier), so they all take the same branch.
__device__ __forceinline__ bool instance_failed(const DevErr* err) {
  return __syncthreads_or(threadIdx.x == 0 && *reinterpret_cast<const volatile int*>(&err->code) != 0) != 0;
}

// ---------------------------------------------------------------------------
// Event keys.
__device__ __forceinline__ uint64_t kpk(uint64_t k) { return k >> 2; }
__device__ __forceinline__ int ktag(uint64_t k) { return int((k >> 2) & 7); }
__device__ __forceinline__ bool kworm(uint64_t k) { return ((k >> 2) & 7) == 7; }
__device__ __forceinline__ int kab(uint64_t k) { return int(k & 1); }
__device__ __forceinline__ int kbl(uint64_t k) { return kworm(k) ? int(1 - (k & 1)) : int((k >> 1) & 1); }
__device__ __forceinline__ int kdir(uint64_t k) { return int((k >> 1) & 1); }
__device__ __forceinline__ uint64_t wkey(uint64_t m, int dir, int above) {
  return (m << 5) | (7ull << 2) | (uint64_t(dir) << 1) | uint64_t(above);
}
// worm grid points strictly between pk a and pk b going up from a (b == a:
// the whole circle); first worm point above / below a vertex point.
__device__ __forceinline__ uint64_t wpts(uint64_t a, uint64_t b) {
  const uint64_t hi = (b > a) ? b : b + kTwo62;
  return (hi >> 3) - ((a + 1) >> 3);
}
__device__ __forceinline__ uint64_t wm_above(uint64_t a) { return ((a + 1) >> 3) & (kTwo59 - 1); }
__device__ __forceinline__ uint64_t wm_below(uint64_t a) { return (((a + 1) >> 3) + kTwo59 - 1) & (kTwo59 - 1); }

// ---------------------------------------------------------------------------
// Temporal domains (Supplement S-II): with N_beta = d.ntau > 1, boundary k of
// every site sits at the grid point m_k = floor(k 2^59 / N_beta) with the
// otherwise unused tag 6, so its time point m_k << 3 | 6 differs from every
// vertex leg and worm; the state there is the worldline's state at that point.
__device__ __forceinline__ uint64_t tb_pk(const Dev& d, int k) {
  const uint64_t kk = uint64_t(k);
  return ((kk * d.tq + (kk * d.tr) / uint64_t(d.ntau)) << 3) | 6u;
}
// pk distance going up from a to b (b == a: the whole circle)
__device__ __forceinline__ uint64_t up_dist(uint64_t a, uint64_t b) {
  return (b == a) ? kTwo62 : ((b - a) & (kTwo62 - 1));
}
// the temporal slab of worm grid point m: the largest k with m_k <= m, i.e.
// k 2^59 < (m + 1) N_beta, k = floor(((m + 1) N_beta - 1) / 2^59) (128-bit)
__device__ __forceinline__ int slab_of_m(const Dev& d, uint64_t m) {
  if (d.ntau < 2) return 0;
  const uint64_t a = m + 1, n = uint64_t(d.ntau);
  uint64_t hi = __umul64hi(a, n), lo = a * n;
  if (lo == 0) hi -= 1;
  lo -= 1;
  return int((hi << 5) | (lo >> 59));
}
// index of the first boundary above pk a / the last one below it (cyclic)
__device__ __forceinline__ int tb_above(const Dev& d, uint64_t a) {
  for (int k = 0; k < d.ntau; ++k) if (tb_pk(d, k) > a) return k;
  return 0;
}
__device__ __forceinline__ int tb_below(const Dev& d, uint64_t a) {
  for (int k = d.ntau - 1; k >= 0; --k) if (tb_pk(d, k) < a) return k;
  return d.ntau - 1;
}

// ---------------------------------------------------------------------------
// Lattice geometry: site i = x + Lx y, bond 2a + d from a to a + x^ / a + y^;
// tag of a bond 3d + cls(c), cls(c) = 2 if c = L-1 else c & 1 (c the
// coordinate of a along d): distinct for the four bonds of a site.
__device__ __forceinline__ int clsf(int c, int L) { return (c == L - 1) ? 2 : (c & 1); }
__device__ __forceinline__ int site_step(const Dev& d, int s, int dir, int sgn) {
  int x = s % d.Lx, y = s / d.Lx;
  if (dir == 0) x = (x + sgn + d.Lx) % d.Lx; else y = (y + sgn + d.Ly) % d.Ly;
  return x + d.Lx * y;
}
__device__ __forceinline__ int bond_tag(const Dev& d, int a, int dir) {
  return dir ? 3 + clsf(a / d.Lx, d.Ly) : clsf(a % d.Lx, d.Lx);
}
// lower site and direction of the bond of a vertex leg with tag t on site s
__device__ __forceinline__ int leg_lower(const Dev& d, int s, int t, int* dir) {
  const int dd = t / 3, cl = t % 3;
  const int c = dd ? s / d.Lx : s % d.Lx, L = dd ? d.Ly : d.Lx;
  *dir = dd;
  return (cl == clsf(c, L)) ? s : site_step(d, s, dd, -1);
}
__device__ __forceinline__ bool boundary_bond(const Dev& d, int a, int dir) {
  if (dir == 0) return d.ndx > 1 && ((a % d.Lx) + 1) % d.dom_x == 0;
  return d.ndy > 1 && ((a / d.Lx) + 1) % d.dom_y == 0;
}
__device__ __forceinline__ int dom_of(const Dev& d, int s) {
  return (s % d.Lx) / d.dom_x + d.ndx * ((s / d.Lx) / d.dom_y);
}

// Step-5 sub-blocks: blocks of B sites at offset 0 or B/2 per axis (periodic
// when one domain spans the axis, clipped at domain edges otherwise).
__device__ __forceinline__ int sb_axis(int c, int D, int B, int nd, int off) {
  if (B == 0 || B >= D) return 0;
  if (nd == 1) return ((c - off + D) % D) / B;
  return (c - off + B) / B;
}
__device__ __forceinline__ int sb_slots(int D, int B, int nd) {
  if (B == 0 || B >= D) return 1;
  return (nd == 1) ? D / B : D / B + 1;
}
__device__ __forceinline__ int sb_local(const Dev& d, int s, int pass) {
  const int B = d.sub_block;
  const int ox = (B && B < d.dom_x) ? (pass & 1) * (B / 2) : 0;
  const int oy = (B && B < d.dom_y) ? ((pass >> 1) & 1) * (B / 2) : 0;
  const int bx = sb_axis((s % d.Lx) % d.dom_x, d.dom_x, B, d.ndx, ox);
  const int by = sb_axis((s / d.Lx) % d.dom_y, d.dom_y, B, d.ndy, oy);
  return bx + sb_slots(d.dom_x, B, d.ndx) * by;
}

// ---------------------------------------------------------------------------
// Per-site event slots: keys sorted by pk in key[s*cap .. s*cap + n).
struct Slot {
  uint64_t* k;
  int n;
};
__device__ __forceinline__ int slot_lower(const uint64_t* k, int n, uint64_t p) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (kpk(k[mid]) < p) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int slot_find(const uint64_t* k, int n, uint64_t p) {
  const int i = slot_lower(k, n, p);
  return (i < n && kpk(k[i]) == p) ? i : -1;
}
// occupation just before time point p (cyclic); base when the slot is empty
__device__ __forceinline__ int slot_state(const uint64_t* k, int n, int base, uint64_t p) {
  if (n == 0) return base;
  const int i = slot_lower(k, n, p);
  return kab(k[(i == 0) ? n - 1 : i - 1]);
}

__device__ __forceinline__ void set_err(DevErr* e, int code, int where) {
  if (atomicCAS(&e->code, 0, code) == 0) e->where = where;
}

}  // namespace pmwa
