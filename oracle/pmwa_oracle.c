/*
 * pmwa_oracle.c -- plain, slow CPU oracle of the PMWA sweep.
 *
 * TEST INFRASTRUCTURE ONLY (see pmwa_oracle.h).  Written for clarity: every
 * site keeps a sorted dynamic array of 64-bit event keys, every random number
 * is recomputed from the Philox counter it belongs to, and the steps run one
 * after the other in canonical order (domains in id order, sites in index
 * order, bonds in index order, worms in label order).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction: every
 * floating-point result must be the IEEE binary64 result of + - * / in the
 * order written).
 *
 * Event key layout (one u64 per event on a site's imaginary-time circle):
 *   bits 63..5  m    time-grid index, 2^59 grid points per beta
 *   bits  4..2  tag  0..5: vertex leg of a bond of class tag (3 d + cls),
 *                    7: worm
 *   bit      1       vertex leg: state just below; worm: direction (1 = up)
 *   bit      0       state just above the event
 * pk = key >> 2 orders the events of a site in time; the tag makes the time
 * points of the bonds meeting at a site and of the worms pairwise disjoint.
 */
#include "pmwa_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define TWO59 ((uint64_t)1 << 59)
#define TWO62 ((uint64_t)1 << 62)
#define TWO32 ((uint64_t)1 << 32)

enum { PH_INIT = 1, PH_BX = 2, PH_BY = 3, PH_VERTEX = 4, PH_REGEN = 5, PH_SCATTER = 6, PH_TEMPORAL = 7 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
   multiply/xor S-box on a 128-bit counter, key bumped by the Weyl constants
   after every round.                                                       */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A stream is the sequence of 64-bit words of the Philox blocks with counter
   (block, unit, c2, sweep); word w is half (w & 1) of block w >> 1.         */
typedef struct {
  uint32_t key[2];
  uint32_t unit, c2, sweep;
  uint64_t pos;
  int      err;
} stream_t;

static uint32_t c2_of(int phase, int pass, uint32_t replica) {
  return (uint32_t)phase | ((uint32_t)pass << 4) | (replica << 16);
}

static void s_init(stream_t* s, uint64_t seed, uint32_t unit, uint32_t c2, uint32_t sweep) {
  s->key[0] = (uint32_t)seed;
  s->key[1] = (uint32_t)(seed >> 32);
  s->unit = unit; s->c2 = c2; s->sweep = sweep; s->pos = 0; s->err = 0;
}

static uint64_t s_word(stream_t* s) {
  uint64_t blk = s->pos >> 1;
  if (blk >= TWO32) s->err = OR_ETIMEOUT;
  uint32_t ctr[4] = { (uint32_t)blk, s->unit, s->c2, s->sweep }, o[4];
  or_philox4x32_10(ctr, s->key, o);
  uint64_t w = (s->pos & 1) ? ((uint64_t)o[2] | ((uint64_t)o[3] << 32))
                            : ((uint64_t)o[0] | ((uint64_t)o[1] << 32));
  s->pos++;
  return w;
}

/* floor(a * b / 2^64): a uniform integer in [0, b) from a uniform u64 a. */
static uint64_t mulhi64(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * b) >> 64); }

/* ------------------------------------------------------------------------ */
/* exp_det: Cody-Waite argument reduction x = k ln2 + r, |r| <= ln2/2, then
   the degree-13 Taylor polynomial of e^r in Horner form, then exact scaling
   by 2^k.  Only IEEE + - * / are used, so the result is the same on every
   conforming machine.  ln2 is split into a 24-bit head (k*LN2_HI exact for
   |k| < 2^29) and the binary64 rounding of the remainder.                   */
static const double INV_LN2 = 1.4426950408889634;      /* 1/ln 2              */
static const double LN2_HI  = 0.693147182464599609375; /* ln 2 rounded to 24 bits */
static const double LN2_LO  = -1.9046542999577678e-09; /* ln 2 - LN2_HI       */

static double ipow2(int k) {           /* 2^k for -1022 <= k <= 1023, exact */
  union { uint64_t u; double d; } v;
  v.u = (uint64_t)(k + 1023) << 52;
  return v.d;
}

double or_exp_det(double x) {
  if (x != x) return x;
  if (x > 709.0) return INFINITY;
  if (x < -745.0) return 0.0;
  double c[14];
  double fact = 1.0;
  for (int n = 0; n <= 13; n++) { if (n > 0) fact = fact * (double)n; c[n] = 1.0 / fact; }
  double kd = floor(x * INV_LN2 + 0.5);
  int k = (int)kd;
  double r = (x - kd * LN2_HI) - kd * LN2_LO;
  double p = c[13];
  for (int n = 12; n >= 0; n--) p = p * r + c[n];
  if (k >= -1022) return p * ipow2(k);
  return (p * ipow2(k + 600)) * ipow2(-600);
}

/* e^x - 1 for |x| <= 1: the Taylor series (Horner, no constant term) cut
   at degree 7, 9, 13 or 19 as |x| <= 2^-6, 2^-4, 2^-2 or 1, which keeps the
   truncation below 2^-57 relative; exp_det(x) - 1 for |x| > 1.             */
double or_expm1_det(double x) {
  if (!(x <= 1.0 && x >= -1.0)) return or_exp_det(x) - 1.0;
  double ax = fabs(x);
  int d = (ax <= 0x1p-6) ? 7 : (ax <= 0x1p-4) ? 9 : (ax <= 0x1p-2) ? 13 : 19;
  double c[20];
  double fact = 1.0;
  for (int n = 1; n <= 19; n++) { fact = fact * (double)n; c[n] = 1.0 / fact; }
  double p = c[d];
  for (int n = d - 1; n >= 1; n--) p = p * x + c[n];
  return p * x;
}

/* tanh x and coth x for x >= 0 from em1 = e^{-2x} - 1:
   tanh x = -em1 / (2 + em1), coth x = (2 + em1) / -em1.                   */
static double tanh_det(double x) { double e = or_expm1_det(-2.0 * x); return -e / (2.0 + e); }
static double coth_det(double x) { double e = or_expm1_det(-2.0 * x); return (2.0 + e) / -e; }

/* ------------------------------------------------------------------------ */
/* Ziggurat for the unit exponential (Marsaglia and Tsang, J. Stat. Softw.
   5(8), 2000): 256 strips of equal area v under f(x) = e^-x.  Strip 0 is the
   rectangle [0,R] x [0,f(R)] plus the tail x > R; strip i >= 1 is the
   rectangle [0, X[i]] x [F[i], F[i+1]] with F[i] = f(X[i]), X[256] = 0.
   R is found by bisection so that the top strip closes with area v.         */
typedef struct {
  double X[257], F[257], W[256];
  uint64_t K[256], XF[256], RF;
  double R, v;
} zig_t;

/* Lay the strips for a trial R.  Returns -1 if R is too small (the strips
   reach the top of the curve early, or the top strip is smaller than v),
   +1 otherwise.                                                             */
static int zig_lay(double R, zig_t* z) {
  double v = (R + 1.0) * exp(-R);
  double X[257], F[257];
  X[1] = R;
  F[1] = exp(-R);
  for (int i = 1; i <= 254; i++) {
    F[i + 1] = F[i] + v / X[i];
    if (!(F[i + 1] < 1.0)) return -1;
    X[i + 1] = -log(F[i + 1]);
  }
  double top = X[255] * (1.0 - F[255]);
  if (top < v) return -1;
  if (z) {
    z->R = R; z->v = v;
    X[0] = v / F[1]; F[0] = 0.0;
    X[256] = 0.0; F[256] = 1.0;
    for (int i = 0; i <= 256; i++) { z->X[i] = X[i]; z->F[i] = F[i]; }
    for (int i = 0; i < 256; i++) {
      z->K[i] = (uint64_t)floor(X[i + 1] / X[i] * 0x1p53);
      z->W[i] = X[i] * 0x1p-53;
      z->XF[i] = (uint64_t)(X[i] * 0x1p58);  /* exact: X[i] has 53 bits, X[i] >= 2^-5 */
    }
    z->RF = (uint64_t)(R * 0x1p58);
  }
  return 1;
}

static void zig_build(zig_t* z) {
  double lo = 7.0, hi = 8.0;
  for (;;) {
    double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (zig_lay(mid, NULL) < 0) lo = mid; else hi = mid;
  }
  zig_lay(hi, z);
}

void or_zig_tables(double* X, double* F, double* W, uint64_t* K, double* R, double* v) {
  zig_t z;
  zig_build(&z);
  memcpy(X, z.X, sizeof z.X); memcpy(F, z.F, sizeof z.F);
  memcpy(W, z.W, sizeof z.W); memcpy(K, z.K, sizeof z.K);
  *R = z.R; *v = z.v;
}

/* One unit exponential deviate E, returned in fixed point as floor-ish
   E 2^58 (u64; E < 64).  A word gives the strip i (low 8 bits) and a 53-bit
   uniform u (high bits); the point is x = u X[i] / 2^53, in fixed point
   (u XF[i]) >> 53 with XF[i] = X[i] 2^58 (exact, 128-bit product).  Inside
   the inner rectangle (u < K[i]) it is accepted at once; strip 0 beyond R
   restarts at R + (new deviate) (memorylessness); otherwise a second word
   places y in the strip and the point is kept if y < e^-x, a binary64 test
   (rare: about 1 % of the words).  At most 64 words.                       */
static uint64_t zfix_add(uint64_t a, uint64_t b) { return (a > UINT64_MAX - b) ? UINT64_MAX : a + b; }

static uint64_t zig_exp(const zig_t* z, stream_t* s) {
  uint64_t acc = 0;
  for (int tries = 0; tries < 64; tries++) {
    uint64_t w = s_word(s);
    unsigned i = (unsigned)(w & 255u);
    uint64_t u = w >> 11;
    uint64_t xf = (uint64_t)(((u128)u * z->XF[i]) >> 53);
    if (u < z->K[i]) return zfix_add(acc, xf);
    if (i == 0) { acc = zfix_add(acc, z->RF); continue; }
    double x = (double)u * z->W[i];
    uint64_t w2 = s_word(s);
    double t1 = (double)(w2 >> 11) * 0x1p-53;
    double t2 = z->F[i + 1] - z->F[i];
    double y = z->F[i] + t1 * t2;
    if (y < or_exp_det(-x)) return zfix_add(acc, xf);
  }
  s->err = OR_ETIMEOUT;
  return 0;
}

int or_exp_deviates(uint64_t seed, uint32_t unit, uint32_t c2, uint32_t sweep,
                    int64_t n, double* out) {
  zig_t z; zig_build(&z);
  stream_t s; s_init(&s, seed, unit, c2, sweep);
  for (int64_t k = 0; k < n; k++) out[k] = (double)zig_exp(&z, &s) * 0x1p-58;
  return s.err;
}

/* A grid scale S (the mean spacing of a Bernoulli process, in grid points)
   as S = m 2^(sh - 122) ... written so that, with E in fixed point (E 2^58),
   E S = (E 2^58) m / 2^sh: m in [2^63, 2^64) is the 53-bit binary64 mantissa
   of S moved to the top of a u64 and sh = 121 - floor(log2 S).  Parameters
   keep S in [2^39, 2^99], so sh stays in [22, 82].                          */
typedef struct { uint64_t m; int sh; } scale_t;

static scale_t scale_of(double S) {
  scale_t r;
  int e;
  double f = frexp(S, &e);          /* S = f 2^e, f in [0.5, 1) */
  r.m = (uint64_t)ldexp(f, 64);     /* exact: f has 53 bits      */
  r.sh = 122 - e;                   /* floor(log2 S) = e - 1     */
  return r;
}

/* Gap of a Bernoulli process on an integer grid with mean spacing S:
   1 + floor(E S) for a unit exponential E (fixed point, 2^-58), from the
   exact 128-bit product; saturates at 2^62.                               */
static uint64_t grid_gap(uint64_t Ef, scale_t S) {
  u128 g = ((u128)Ef * S.m) >> S.sh;
  if (g >= (u128)TWO62) return TWO62;
  return 1 + (uint64_t)g;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 for hard-core bosons: the number of worms n on an interval has
   P(n) proportional to x^n / n! restricted to n = sigma (mod 2), where
   x = I eta and sigma is the parity of the interval (its end states differ),
   and the n worm times are uniform.  Equivalently: a rate-eta Poisson process
   on the interval conditioned on the parity of its count.  The interval is
   the M worm grid points strictly inside it; SW = 2^59 / (beta eta) is the
   mean grid spacing of the process.
     sigma = 0, or sigma = 1 with x > 1: draw the process, keep it if the
       parity is right (acceptance >= 0.43), else draw again;
     sigma = 1 with x <= 1 (M <= SWI = floor(SW)): propose n = 1 + (count of
       the process), keep it with probability 1/n if n is odd, the extra
       worm at a uniform grid point (a clash with a process point is a
       rejection).  This gives x^n/n! for odd n; acceptance >= 0.43.
   At most 128 proposals.  Offsets (0 <= off < M) are written sorted.       */
static int sample_worms(const zig_t* z, stream_t* s, uint64_t M, int sigma,
                        scale_t SW, uint64_t SWI, uint64_t* offs, int max) {
  if (M == 0) { if (sigma) { s->err = OR_EINVARIANT; return -1; } return 0; }
  for (int tries = 0; tries < 128; tries++) {
    int n = 0, first = 1;
    uint64_t pos = 0;
    for (;;) {
      uint64_t E = zig_exp(z, s);
      uint64_t g = grid_gap(E, SW);
      uint64_t nxt = first ? g - 1 : pos + g;
      first = 0;
      if (nxt >= M) break;
      pos = nxt;
      if (n >= max) { s->err = OR_ETIMEOUT; return -1; }
      offs[n++] = pos;
    }
    if (sigma == 1 && M <= SWI) {
      int ntot = n + 1;
      if ((ntot & 1) == 0) continue;
      if (mulhi64(s_word(s), (uint64_t)ntot) != 0) continue;
      uint64_t extra = mulhi64(s_word(s), M);
      int clash = 0, at = n;
      for (int k = 0; k < n; k++) {
        if (offs[k] == extra) { clash = 1; break; }
        if (offs[k] > extra) { at = k; break; }
      }
      if (clash) continue;
      if (n >= max) { s->err = OR_ETIMEOUT; return -1; }
      for (int k = n; k > at; k--) offs[k] = offs[k - 1];
      offs[at] = extra;
      return ntot;
    }
    if ((n & 1) == sigma) return n;
  }
  s->err = OR_ETIMEOUT;
  return -1;
}

static uint64_t swi_of(double SW) { return (SW >= 0x1p62) ? TWO62 : (uint64_t)SW; }

int or_sample_worms(uint64_t seed, uint32_t unit, uint32_t c2, uint32_t sweep,
                    uint64_t M, int sigma, double SW, uint64_t* offs, int max) {
  static zig_t z;
  static int built = 0;
  if (!built) { zig_build(&z); built = 1; }
  stream_t s; s_init(&s, seed, unit, c2, sweep);
  int n = sample_worms(&z, &s, M, sigma, scale_of(SW), swi_of(SW), offs, max);
  return s.err ? -1 : n;
}

/* ------------------------------------------------------------------------ */
/* Configuration: per site a sorted array of event keys, a parallel array of
   worm labels (meaningful for worms only, Step 4 -> Step 5), and the state
   at the start of the circle (needed when the site has no events).        */
typedef struct {
  uint64_t* key;
  uint64_t* lab;
  int n, cap;
  int base;
} site_t;

struct or_handle {
  or_params p;
  int N, Lx, Ly, ndx, ndy, ndom, K;
  double d[4], D, C, SV, SW;
  scale_t SVs, SWs;
  uint64_t TV[4], SWI;
  uint64_t TH[16][4][4];
  zig_t z;
  site_t* site;
  uint64_t sweep;
  or_row* rows; int64_t nrows, caprows;
  int err;
};

static inline uint64_t kpk(uint64_t k) { return k >> 2; }
static inline int ktag(uint64_t k) { return (int)((k >> 2) & 7); }
static inline int kworm(uint64_t k) { return ktag(k) == 7; }
static inline int kab(uint64_t k) { return (int)(k & 1); }                 /* state above */
static inline int kbl(uint64_t k) { return kworm(k) ? (int)(1 - (k & 1)) : (int)((k >> 1) & 1); }
static inline int kdir(uint64_t k) { return (int)((k >> 1) & 1); }

static void site_reserve(site_t* s, int n) {
  if (n <= s->cap) return;
  int c = s->cap ? s->cap : 16;
  while (c < n) c *= 2;
  s->key = (uint64_t*)realloc(s->key, sizeof(uint64_t) * (size_t)c);
  s->lab = (uint64_t*)realloc(s->lab, sizeof(uint64_t) * (size_t)c);
  s->cap = c;
}
static void site_insert(site_t* s, int at, uint64_t key, uint64_t lab) {
  site_reserve(s, s->n + 1);
  memmove(s->key + at + 1, s->key + at, sizeof(uint64_t) * (size_t)(s->n - at));
  memmove(s->lab + at + 1, s->lab + at, sizeof(uint64_t) * (size_t)(s->n - at));
  s->key[at] = key; s->lab[at] = lab; s->n++;
}
static void site_erase(site_t* s, int at) {
  memmove(s->key + at, s->key + at + 1, sizeof(uint64_t) * (size_t)(s->n - at - 1));
  memmove(s->lab + at, s->lab + at + 1, sizeof(uint64_t) * (size_t)(s->n - at - 1));
  s->n--;
}
/* index of the first event with pk >= p (n if none) */
static int site_lower(const site_t* s, uint64_t p) {
  int i = 0;
  while (i < s->n && kpk(s->key[i]) < p) i++;
  return i;
}
static int site_find(const site_t* s, uint64_t p) {
  int i = site_lower(s, p);
  return (i < s->n && kpk(s->key[i]) == p) ? i : -1;
}
/* insert keeping the array sorted by key */
static void site_add(site_t* s, uint64_t key, uint64_t lab) { site_insert(s, site_lower(s, kpk(key)), key, lab); }

/* occupation just before time point p (cyclic): state above the last event
   with pk < p, else above the last event of the circle, else the base.   */
static int state_at(const site_t* s, uint64_t p) {
  if (s->n == 0) return s->base;
  int i = site_lower(s, p);
  return kab(s->key[(i == 0) ? s->n - 1 : i - 1]);
}
static void fix_base(site_t* s) { if (s->n) s->base = kab(s->key[s->n - 1]); }

/* worm grid points strictly between pk a and pk b, going up from a (cyclic);
   b == a means the whole circle.                                          */
static uint64_t wpts(uint64_t a, uint64_t b) {
  uint64_t hi = (b > a) ? b : b + TWO62;
  return (hi >> 3) - ((a + 1) >> 3);
}
/* m of the first worm grid point above pk a, and of the first one below. */
static uint64_t wm_above(uint64_t a) { return ((a + 1) >> 3) & (TWO59 - 1); }
static uint64_t wm_below(uint64_t a) { return (((a + 1) >> 3) + TWO59 - 1) & (TWO59 - 1); }
static uint64_t wkey(uint64_t m, int dir, int above) {
  return (m << 5) | (7u << 2) | ((uint64_t)dir << 1) | (uint64_t)above;
}

/* ------------------------------------------------------------------------ */
/* Temporal domains (Supplement S-II: the space-time is cut into N_beta
   slabs along imaginary time; Step 1 and Eq. 3).  With N_beta = dom_tau > 1
   boundary k (k = 0..N_beta-1) sits on every site at the grid point
   m_k = floor(k 2^59 / N_beta) with the otherwise unused tag 6, so its time
   point tb_pk(k) = m_k << 3 | 6 is distinct from every vertex leg and worm.
   A boundary is no event of the configuration: the state there is the state
   of the worldline at that point, which only Step 1 changes (Steps 2, 4 and
   5 stop at boundaries and keep the parity of every piece).  With
   N_beta = 1 there is no boundary.                                        */
static int ntau(const or_handle* h) { return h->p.dom_tau; }
static uint64_t tb_pk(const or_handle* h, int k) {
  uint64_t m = (uint64_t)(((u128)(uint64_t)k << 59) / (u128)(uint64_t)h->p.dom_tau);
  return (m << 3) | 6u;
}
/* pk distance going up from a to b (b == a: the whole circle, 2^62) */
static uint64_t up_dist(uint64_t a, uint64_t b) { return (b == a) ? TWO62 : ((b - a) & (TWO62 - 1)); }
/* the first boundary above pk a, and the last one below it (cyclic) */
static int tb_above(const or_handle* h, uint64_t a) {
  for (int k = 0; k < ntau(h); k++) if (tb_pk(h, k) > a) return k;
  return 0;
}
static int tb_below(const or_handle* h, uint64_t a) {
  for (int k = ntau(h) - 1; k >= 0; k--) if (tb_pk(h, k) < a) return k;
  return ntau(h) - 1;
}
/* a boundary strictly between pk a and pk b going up from a (b == a: the
   whole circle but a) */
static int tb_between(const or_handle* h, uint64_t a, uint64_t b) {
  if (ntau(h) < 2) return 0;
  return up_dist(a, tb_pk(h, tb_above(h, a))) < up_dist(a, b);
}
/* the temporal slab of a worm at pk w: the index of the last boundary below */
static int slab_of(const or_handle* h, uint64_t w) { return ntau(h) < 2 ? 0 : tb_below(h, w); }

/* ------------------------------------------------------------------------ */
/* Geometry.  Site i = x + Lx y; bond b = 2 a + d joins its lower site a to
   a + x^ (d = 0) or a + y^ (d = 1), periodic.  Legs of a vertex: 0 = a below,
   1 = upper site below, 2 = a above, 3 = upper site above.  A bond's tag is
   3 d + cls(c), c the coordinate of a along d, cls(c) = 2 if c = L-1 else
   c mod 2: the four bonds meeting at a site get four different tags for
   every L >= 2, so the tag of a vertex leg names its bond.                  */
static int sx(const or_handle* h, int s) { return s % h->Lx; }
static int sy(const or_handle* h, int s) { return s / h->Lx; }
static int step(const or_handle* h, int s, int d, int sgn) {
  int x = sx(h, s), y = sy(h, s);
  if (d == 0) x = (x + sgn + h->Lx) % h->Lx; else y = (y + sgn + h->Ly) % h->Ly;
  return x + h->Lx * y;
}
static int clsf(int c, int L) { return (c == L - 1) ? 2 : (c & 1); }
static int bond_tag(const or_handle* h, int a, int d) {
  return 3 * d + (d ? clsf(sy(h, a), h->Ly) : clsf(sx(h, a), h->Lx));
}
/* bond of the vertex leg with tag t on site s: its lower site and direction */
static void leg_bond(const or_handle* h, int s, int t, int* a, int* d) {
  int dd = t / 3, cl = t % 3;
  int c = dd ? sy(h, s) : sx(h, s), L = dd ? h->Ly : h->Lx;
  *d = dd;
  *a = (cl == clsf(c, L)) ? s : step(h, s, dd, -1);
}
static int dom_of(const or_handle* h, int s) {
  return sx(h, s) / h->p.dom_x + h->ndx * (sy(h, s) / h->p.dom_y);
}
/* a bond whose two sites lie in different domains (Step 2 handles it) */
static int is_boundary_bond(const or_handle* h, int a, int d) {
  if (d == 0) return h->ndx > 1 && (sx(h, a) + 1) % h->p.dom_x == 0;
  return h->ndy > 1 && (sy(h, a) + 1) % h->p.dom_y == 0;
}

/* Shifted sub-block schedule of Step 5.  Along an axis with domain extent D
   and edge B: one block if B == 0 or B >= D; else blocks of B sites starting
   at offset off = 0 or B/2, periodic when the domain spans the lattice along
   that axis, clipped at the domain edges otherwise.                        */
static int sb_axis(int c, int D, int B, int nd, int off) {
  if (B == 0 || B >= D) return 0;
  if (nd == 1) return ((c - off + D) % D) / B;
  return (c - off + B) / B;
}
static int sb_slots(int D, int B, int nd) {
  if (B == 0 || B >= D) return 1;
  return (nd == 1) ? D / B : D / B + 1;
}
static void sb_offsets(const or_handle* h, int pass, int* ox, int* oy) {
  int B = h->p.sub_block;
  *ox = (B && B < h->p.dom_x) ? (pass & 1) * (B / 2) : 0;
  *oy = (B && B < h->p.dom_y) ? ((pass >> 1) & 1) * (B / 2) : 0;
}
/* global id of the sub-block holding site s in pass `pass` */
static uint32_t sb_unit(const or_handle* h, int s, int pass) {
  int ox, oy; sb_offsets(h, pass, &ox, &oy);
  int B = h->p.sub_block, Dx = h->p.dom_x, Dy = h->p.dom_y;
  int bx = sb_axis(sx(h, s) % Dx, Dx, B, h->ndx, ox);
  int by = sb_axis(sy(h, s) % Dy, Dy, B, h->ndy, oy);
  int nx = sb_slots(Dx, B, h->ndx), ny = sb_slots(Dy, B, h->ndy);
  return (uint32_t)(dom_of(h, s) * nx * ny + bx + nx * by);
}
/* a bond whose vertices a worm may enter in this pass */
static int bond_active(const or_handle* h, int a, int d, int pass) {
  if (is_boundary_bond(h, a, d)) return 0;
  return sb_unit(h, a, pass) == sb_unit(h, step(h, a, d, +1), pass);
}

/* ------------------------------------------------------------------------ */
/* Model (Eq. 5 per bond): E(na,nb) = V na nb - (mu/4)(na + nb).  Vertex
   weights (Step 3 density, Eq. 2 w_i): diagonal d(s) = C - E(s) with
   C = max E + c_off; kink t.  D = max d is the candidate rate of Step 3;
   a candidate in state s is kept with probability d(s)/D (thinning).     */
static double vweight(const or_handle* h, int S) {
  int s0 = S & 1, s1 = (S >> 1) & 1, s2 = (S >> 2) & 1, s3 = (S >> 3) & 1;
  if (s0 + s1 != s2 + s3) return 0.0;
  if (s0 == s2) return h->d[s0 | (s1 << 1)];
  return h->p.t;
}

/* Directed-loop solution of one scattering family (weights w[0..3] of the
   states with the worm on leg l): sort the positive weights a >= b >= c
   (missing ones count as 0); if a <= b + c there is no bounce,
   w_ab = (a+b-c)/2, w_ac = (a+c-b)/2, w_bc = (b+c-a)/2; otherwise
   w_aa = a-b-c, w_ab = b, w_ac = c.  Fills m[l][l'] (symmetric).         */
static void dl_solve(const double w[4], double m[4][4]) {
  int ord[4] = {0, 1, 2, 3};
  for (int i = 0; i < 4; i++)            /* stable sort, descending weight */
    for (int j = 3; j > i; j--)
      if (w[ord[j]] > w[ord[j - 1]]) { int t = ord[j]; ord[j] = ord[j - 1]; ord[j - 1] = t; }
  for (int i = 0; i < 4; i++) for (int j = 0; j < 4; j++) m[i][j] = 0.0;
  int ia = ord[0], ib = ord[1], ic = ord[2];
  double a = w[ia], b = w[ib], c = w[ic];
  if (a <= b + c) {
    m[ia][ib] = m[ib][ia] = ((a + b) - c) / 2.0;
    m[ia][ic] = m[ic][ia] = ((a + c) - b) / 2.0;
    m[ib][ic] = m[ic][ib] = ((b + c) - a) / 2.0;
  } else {
    m[ia][ia] = (a - b) - c;
    m[ia][ib] = m[ib][ia] = b;
    m[ia][ic] = m[ic][ia] = c;
  }
}

static int derive(or_handle* h) {
  const or_params* p = &h->p;
  double c_off = (p->c_off < 0.0) ? 0.5 * p->t : p->c_off;
  double E[4], Emax = -INFINITY;
  for (int s = 0; s < 4; s++) {
    int na = s & 1, nb = s >> 1;
    E[s] = p->V * (double)(na * nb) - (p->mu / 4.0) * (double)(na + nb);
    if (E[s] > Emax) Emax = E[s];
  }
  h->C = Emax + c_off;
  h->D = 0.0;
  for (int s = 0; s < 4; s++) { h->d[s] = h->C - E[s]; if (h->d[s] > h->D) h->D = h->d[s]; }
  for (int s = 0; s < 4; s++)
    h->TV[s] = (h->d[s] == h->D) ? TWO32 : (uint64_t)floor(h->d[s] / h->D * 0x1p32);
  h->SV = (h->D > 0.0) ? 0x1p59 / (p->beta * h->D) : INFINITY;
  h->SW = 0x1p59 / (p->beta * p->eta);
  h->SWI = swi_of(h->SW);
  h->SWs = scale_of(h->SW);
  if (h->D > 0.0) h->SVs = scale_of(h->SV);
  for (int S = 0; S < 16; S++)
    for (int i = 0; i < 4; i++) {
      double wi = vweight(h, S);
      for (int j = 0; j < 4; j++) h->TH[S][i][j] = TWO32;
      if (wi <= 0.0) continue;
      int T = S ^ (1 << i);
      double w[4], m[4][4];
      for (int l = 0; l < 4; l++) w[l] = vweight(h, T ^ (1 << l));
      dl_solve(w, m);
      int last = 0;
      for (int j = 0; j < 4; j++) if (m[i][j] > 0.0) last = j;
      double cum = 0.0;
      for (int j = 0; j < 4; j++) {
        cum = cum + m[i][j] / wi;
        h->TH[S][i][j] = (j >= last) ? TWO32 : (uint64_t)floor(cum * 0x1p32);
      }
    }
  return OR_OK;
}

int or_tables(const or_params* p, double* d4, double* Dmax, uint64_t* TV4,
              uint64_t* TH256, double* SV, double* SW) {
  or_handle h; memset(&h, 0, sizeof h);
  h.p = *p;
  derive(&h);
  for (int s = 0; s < 4; s++) { d4[s] = h.d[s]; TV4[s] = h.TV[s]; }
  *Dmax = h.D; *SV = h.SV; *SW = h.SW;
  memcpy(TH256, h.TH, sizeof h.TH);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 3 (vertex phase) on one bond: erase its diagonal vertices, keep its
   kinks, and lay new diagonal vertices as a Bernoulli process of mean grid
   spacing SV = 2^59/(beta D) on the bond's 2^59 time points, each kept with
   probability d(s)/D, s the pair of occupations at that time (a point held
   by a kink of the bond is skipped).  Diagonal vertices never change the
   occupations, so every bond may be treated in any order.                 */
/* On-the-fly vertex generation (the paper's closing discussion of
   extensions: vertices generated only near the worms).  With
   vertex_window = w > 0 the vertex phase of a bond is confined to the region
   R of time points within w beta of a worm on either of its two sites (worm
   grid points, cyclic): only the diagonal vertices inside R are erased, and
   only the candidates inside R are placed.  R depends on the worms alone,
   which Step 3 does not move, and a Poisson process on R is independent of
   the one outside, so drawing it afresh on R given the rest keeps the
   distribution; Step 4 puts worms anywhere, so every region is reached.
   The window is a fraction of beta, held as worm grid points.              */
typedef struct { uint64_t* m; int n; uint64_t half; } window_t;

static void window_of(const or_handle* h, const site_t* A, const site_t* B, window_t* W) {
  W->n = 0;
  W->m = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(A->n + B->n + 1));
  for (int k = 0; k < A->n; k++) if (kworm(A->key[k])) W->m[W->n++] = kpk(A->key[k]) >> 3;
  for (int k = 0; k < B->n; k++) if (kworm(B->key[k])) W->m[W->n++] = kpk(B->key[k]) >> 3;
  double w = h->p.vertex_window;
  W->half = (w >= 0.5) ? TWO59 : (uint64_t)(w * 0x1p59);
}
/* is grid point pos within the window of a worm (cyclic distance)? */
static int in_window(const window_t* W, uint64_t pos) {
  for (int i = 0; i < W->n; i++) {
    uint64_t d = (pos - W->m[i]) & (TWO59 - 1), e = (W->m[i] - pos) & (TWO59 - 1);
    if ((d < e ? d : e) <= W->half) return 1;
  }
  return 0;
}

static int step3_bond(or_handle* h, int a, int d) {
  int bs = step(h, a, d, +1), tag = bond_tag(h, a, d);
  site_t *A = &h->site[a], *B = &h->site[bs];
  window_t W = { NULL, 0, 0 };
  const int otf = h->p.vertex_window > 0.0;
  if (otf) window_of(h, A, B, &W);
  for (int k = A->n - 1; k >= 0; k--) {
    uint64_t key = A->key[k];
    if (ktag(key) != tag || kab(key) != kbl(key)) continue;
    if (otf && !in_window(&W, kpk(key) >> 3)) continue;  /* kept outside the window */
    uint64_t pk = kpk(key);
    site_erase(A, k);
    int kb = site_find(B, pk);
    if (kb < 0) { free(W.m); return OR_EINVARIANT; }
    site_erase(B, kb);
  }
  if (!(h->D > 0.0)) { free(W.m); return OR_OK; }
  stream_t s;
  s_init(&s, h->p.seed, (uint32_t)(2 * a + d), c2_of(PH_VERTEX, 0, h->p.replica), (uint32_t)h->sweep);
  uint64_t pos = 0;
  int first = 1;
  for (;;) {
    uint64_t E = zig_exp(&h->z, &s);
    uint64_t g = grid_gap(E, h->SVs);
    uint64_t nxt = first ? g - 1 : pos + g;
    first = 0;
    if (nxt >= TWO59) break;
    pos = nxt;
    uint64_t pk = (pos << 3) | (uint64_t)tag;
    if (otf && !in_window(&W, pos)) continue;
    if (site_find(A, pk) >= 0) continue;
    int na = state_at(A, pk), nb = state_at(B, pk);
    int si = na | (nb << 1);
    if (h->TV[si] < TWO32) {
      uint64_t w = s_word(&s);
      if ((w >> 32) >= h->TV[si]) continue;
    }
    site_add(A, (pk << 2) | ((uint64_t)na << 1) | (uint64_t)na, 0);
    site_add(B, (pk << 2) | ((uint64_t)nb << 1) | (uint64_t)nb, 0);
  }
  free(W.m);
  return s.err;
}

#define MAXW 4096
typedef struct { uint64_t key, lab; } ev_t;
static int ev_cmp(const void* x, const void* y) {
  uint64_t a = ((const ev_t*)x)->key, b = ((const ev_t*)y)->key;
  return (a < b) ? -1 : (a > b);
}

/* Step 4 (worm creation) on one site: erase its worms; on every interval
   between consecutive vertex legs (the last one wraps round the circle) draw
   the worms with the Eq. 1 sampler, their types alternating from the state p
   just above the lower leg.  A site without legs is one closed interval of
   length beta: its state is drawn uniformly (both weigh cosh(beta eta)) and
   n is even.  Each new worm then takes one word: label = word >> 1 (its
   place in the Step-5 order), direction = word & 1.
   With temporal domains the intervals are delimited by the vertex legs and
   the temporal boundaries (pseudo code Step 4), each boundary carrying the
   state the worldline has there before the worms are erased; the intervals
   are taken in time order from the lowest delimiter.                       */
static int step4_site_tau(or_handle* h, int si) {
  site_t* S = &h->site[si];
  const int NB = ntau(h);
  int bs[64];
  for (int k = 0; k < NB; k++) bs[k] = state_at(S, tb_pk(h, k));
  int nl = 0;
  for (int k = 0; k < S->n; k++) if (!kworm(S->key[k])) { S->key[nl] = S->key[k]; S->lab[nl] = 0; nl++; }
  S->n = nl;
  /* delimiters in time order: the legs and the boundaries (as keys of tag 6
     whose state below and above is the boundary's state) */
  int nd = nl + NB;
  uint64_t* dl = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nd);
  for (int k = 0; k < nl; k++) dl[k] = S->key[k];
  for (int k = 0; k < NB; k++) dl[nl + k] = (tb_pk(h, k) << 2) | ((uint64_t)bs[k] << 1) | (uint64_t)bs[k];
  for (int i = 1; i < nd; i++)  /* insertion sort by time */
    for (int j = i; j > 0 && kpk(dl[j]) < kpk(dl[j - 1]); j--) { uint64_t t = dl[j]; dl[j] = dl[j - 1]; dl[j - 1] = t; }
  stream_t st;
  s_init(&st, h->p.seed, (uint32_t)si, c2_of(PH_REGEN, 0, h->p.replica), (uint32_t)h->sweep);
  static uint64_t offs[MAXW];
  ev_t* out = (ev_t*)malloc(sizeof(ev_t) * (size_t)(nl + NB * MAXW + 1));
  int no = 0;
  for (int k = 0; k < nd; k++) {
    uint64_t lo = dl[k], hi = dl[(k + 1) % nd];
    if (ktag(lo) != 6) { out[no].key = lo; out[no].lab = 0; no++; }
    uint64_t M = wpts(kpk(lo), kpk(hi));
    int p = kab(lo), sigma = p ^ kbl(hi);
    int n = sample_worms(&h->z, &st, M, sigma, h->SWs, h->SWI, offs, MAXW);
    if (n < 0) { free(out); free(dl); return st.err ? st.err : OR_ETIMEOUT; }
    uint64_t m0 = wm_above(kpk(lo));
    for (int j = 0; j < n; j++) {
      uint64_t w = s_word(&st);
      out[no].key = wkey((m0 + offs[j]) & (TWO59 - 1), (int)(w & 1), p ^ 1 ^ (j & 1));
      out[no].lab = w >> 1;
      no++;
    }
  }
  qsort(out, (size_t)no, sizeof(ev_t), ev_cmp);
  site_reserve(S, no);
  for (int k = 0; k < no; k++) { S->key[k] = out[k].key; S->lab[k] = out[k].lab; }
  S->n = no;
  if (no) fix_base(S); else S->base = bs[0];
  free(out);
  free(dl);
  return st.err;
}

static int step4_site(or_handle* h, int si) {
  if (ntau(h) > 1) return step4_site_tau(h, si);
  site_t* S = &h->site[si];
  int nl = 0;
  for (int k = 0; k < S->n; k++) if (!kworm(S->key[k])) { S->key[nl] = S->key[k]; S->lab[nl] = 0; nl++; }
  S->n = nl;
  stream_t st;
  s_init(&st, h->p.seed, (uint32_t)si, c2_of(PH_REGEN, 0, h->p.replica), (uint32_t)h->sweep);
  static uint64_t offs[MAXW];
  ev_t* out = (ev_t*)malloc(sizeof(ev_t) * (size_t)(nl + MAXW + 1));
  int no = 0;
  if (nl == 0) {
    int s0 = (int)(s_word(&st) >> 63);
    int n = sample_worms(&h->z, &st, TWO59, 0, h->SWs, h->SWI, offs, MAXW);
    if (n < 0) { free(out); return st.err ? st.err : OR_ETIMEOUT; }
    for (int k = 0; k < n; k++) {
      uint64_t w = s_word(&st);
      out[no].key = wkey(offs[k], (int)(w & 1), s0 ^ 1 ^ (k & 1));
      out[no].lab = w >> 1;
      no++;
    }
    S->base = s0;
  } else {
    for (int k = 0; k < nl; k++) {
      uint64_t lo = S->key[k], hi = S->key[(k + 1) % nl];
      out[no].key = lo; out[no].lab = 0; no++;
      uint64_t M = wpts(kpk(lo), kpk(hi));
      int p = kab(lo), sigma = p ^ kbl(hi);
      int n = sample_worms(&h->z, &st, M, sigma, h->SWs, h->SWI, offs, MAXW);
      if (n < 0) { free(out); return st.err ? st.err : OR_ETIMEOUT; }
      uint64_t m0 = wm_above(kpk(lo));
      for (int j = 0; j < n; j++) {
        uint64_t w = s_word(&st);
        out[no].key = wkey((m0 + offs[j]) & (TWO59 - 1), (int)(w & 1), p ^ 1 ^ (j & 1));
        out[no].lab = w >> 1;
        no++;
      }
    }
  }
  qsort(out, (size_t)no, sizeof(ev_t), ev_cmp);
  site_reserve(S, no);
  for (int k = 0; k < no; k++) { S->key[k] = out[k].key; S->lab[k] = out[k].lab; }
  S->n = no;
  fix_base(S);
  free(out);
  return st.err;
}

/* length (worm grid points) of the leg of the vertex at pk pv on site x,
   upward or downward, up to the next event other than the skipped worm;
   the whole circle (2^59) if there is none.  With temporal domains a leg
   also ends at the next temporal boundary (Eq. 2 within a domain).        */
static uint64_t leg_len(const or_handle* h, int x, uint64_t pv, int up, int skip_site, uint64_t skip_pk) {
  const site_t* S = &h->site[x];
  int iv = site_find(S, pv), n = S->n, j = iv;
  uint64_t len = TWO59;
  for (int k = 0; k < n; k++) {
    j = up ? (j + 1) % n : (j + n - 1) % n;
    if (j == iv) break;
    uint64_t pj = kpk(S->key[j]);
    if (x == skip_site && pj == skip_pk) continue;
    len = up ? wpts(pv, pj) : wpts(pj, pv);
    break;
  }
  if (ntau(h) > 1) {
    uint64_t lb = up ? wpts(pv, tb_pk(h, tb_above(h, pv))) : wpts(tb_pk(h, tb_below(h, pv)), pv);
    if (lb < len) len = lb;
  }
  return len;
}

static void flip_leg_bit(or_handle* h, int x, uint64_t pv, int below) {
  site_t* S = &h->site[x];
  int k = site_find(S, pv);
  S->key[k] ^= below ? 2u : 1u;
}

/* Step 5: one move of the worm at (ws, wpk), with the two words of its Philox
   block.  Nearest event ahead: a worm, or a vertex whose bond is not active
   in this pass (domain or sub-block edge), makes it turn round in place.
   Otherwise the worm on leg i enters the vertex with probability L_min/L_i
   (u32 of word0 >> 32 against the exact ratio), leaves by leg j with the
   directed-loop threshold table (u32 of word0), and lands at a uniform grid
   point of leg j (mulhi of word1), heading away from the vertex (Eq. 2).   */
static int scatter_move(or_handle* h, int pass, int ws, uint64_t wpk, uint64_t w0, uint64_t w1) {
  site_t* S = &h->site[ws];
  int iw = site_find(S, wpk);
  if (iw < 0 || S->n < 2) return OR_EINVARIANT;
  uint64_t key = S->key[iw], lab = S->lab[iw];
  int up = kdir(key), n = S->n;
  int ie = up ? (iw + 1) % n : (iw + n - 1) % n;
  uint64_t ke = S->key[ie];
  if (kworm(ke)) { S->key[iw] ^= 2u; return OR_OK; }
  /* a temporal boundary before the next event turns it round (pseudo code Step 5) */
  if (tb_between(h, up ? wpk : kpk(ke), up ? kpk(ke) : wpk)) { S->key[iw] ^= 2u; return OR_OK; }
  int a, d;
  leg_bond(h, ws, ktag(ke), &a, &d);
  if (!bond_active(h, a, d, pass)) { S->key[iw] ^= 2u; return OR_OK; }
  int b = step(h, a, d, +1);
  uint64_t pv = kpk(ke);
  int i = (ws == a) ? (up ? 0 : 2) : (up ? 1 : 3);
  uint64_t L[4], Lmin = 0;
  for (int l = 0; l < 4; l++) {
    L[l] = leg_len(h, (l & 1) ? b : a, pv, l >= 2, ws, wpk);
    if (l == 0 || L[l] < Lmin) Lmin = L[l];
  }
  uint64_t z1 = w0 >> 32, z0 = w0 & 0xffffffffu;
  if (!((u128)z1 * L[i] < ((u128)Lmin << 32))) { S->key[iw] ^= 2u; return OR_OK; }
  const site_t *A = &h->site[a], *Bs = &h->site[b];
  uint64_t va = A->key[site_find(A, pv)], vb = Bs->key[site_find(Bs, pv)];
  int Sst = kbl(va) | (kbl(vb) << 1) | (kab(va) << 2) | (kab(vb) << 3);
  int j = 0;
  while (j < 3 && !(z0 < h->TH[Sst][i][j])) j++;
  site_erase(S, iw);
  flip_leg_bit(h, (i & 1) ? b : a, pv, i < 2);
  flip_leg_bit(h, (j & 1) ? b : a, pv, j < 2);
  int x = (j & 1) ? b : a;
  const site_t* X = &h->site[x];
  uint64_t vx = X->key[site_find(X, pv)];
  uint64_t o = mulhi64(w1, L[j]);
  uint64_t nk;
  if (j >= 2) nk = wkey((wm_above(pv) + o) & (TWO59 - 1), 1, kab(vx) ^ 1);
  else        nk = wkey((wm_below(pv) + TWO59 - o) & (TWO59 - 1), 0, kbl(vx));
  site_add(&h->site[x], nk, lab);
  fix_base(&h->site[a]);
  fix_base(&h->site[b]);
  return OR_OK;
}

typedef struct { int site; uint64_t pk, lab; } wref_t;
static int wref_cmp(const void* x, const void* y) {
  const wref_t *a = (const wref_t*)x, *b = (const wref_t*)y;
  if (a->lab != b->lab) return (a->lab < b->lab) ? -1 : 1;
  if (a->site != b->site) return (a->site < b->site) ? -1 : 1;
  return (a->pk < b->pk) ? -1 : (a->pk > b->pk);
}

/* One Step-5 pass: every sub-block (in unit order) moves each of its worms
   once, in ascending label order; the r-th move uses Philox block r of the
   stream (unit = sub-block id, c2 = scatter | pass).  With temporal domains
   the unit is a sub-block of one slab, sub-block id * N_beta + slab: a worm
   never leaves its slab (it turns round at the boundaries and every leg
   ends there), so the slabs of a sub-block are independent chains.        */
static uint32_t worm_unit(const or_handle* h, uint32_t sb, uint64_t wpk) {
  return sb * (uint32_t)ntau(h) + (uint32_t)slab_of(h, wpk);
}

static int step5_pass(or_handle* h, int pass) {
  int N = h->N;
  uint32_t* unit = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  uint32_t umax = 0;
  for (int s = 0; s < N; s++) { unit[s] = sb_unit(h, s, pass); if (unit[s] > umax) umax = unit[s]; }
  umax = (umax + 1) * (uint32_t)ntau(h) - 1;
  int64_t nw = 0;
  for (int s = 0; s < N; s++) for (int k = 0; k < h->site[s].n; k++) nw += kworm(h->site[s].key[k]);
  wref_t* W = (wref_t*)malloc(sizeof(wref_t) * (size_t)(nw + 1));
  /* bucket the worms by sub-block */
  int64_t* cnt = (int64_t*)calloc((size_t)umax + 2, sizeof(int64_t));
  for (int s = 0; s < N; s++)
    for (int k = 0; k < h->site[s].n; k++)
      if (kworm(h->site[s].key[k])) cnt[worm_unit(h, unit[s], kpk(h->site[s].key[k])) + 1]++;
  for (uint32_t u = 0; u <= umax; u++) cnt[u + 1] += cnt[u];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)umax + 1));
  for (uint32_t u = 0; u <= umax; u++) fill[u] = cnt[u];
  for (int s = 0; s < N; s++)
    for (int k = 0; k < h->site[s].n; k++)
      if (kworm(h->site[s].key[k])) {
        wref_t r = { s, kpk(h->site[s].key[k]), h->site[s].lab[k] };
        W[fill[worm_unit(h, unit[s], r.pk)]++] = r;
      }
  int rc = OR_OK;
  for (uint32_t u = 0; u <= umax && rc == OR_OK; u++) {
    int64_t lo = cnt[u], hi = cnt[u + 1];
    qsort(W + lo, (size_t)(hi - lo), sizeof(wref_t), wref_cmp);
    stream_t st;
    s_init(&st, h->p.seed, u, c2_of(PH_SCATTER, pass, h->p.replica), (uint32_t)h->sweep);
    for (int64_t r = 0; r < hi - lo && rc == OR_OK; r++) {
      st.pos = 2 * (uint64_t)r;
      uint64_t w0 = s_word(&st), w1 = s_word(&st);
      rc = scatter_move(h, pass, W[lo + r].site, W[lo + r].pk, w0, w1);
    }
  }
  free(unit); free(W); free(cnt); free(fill);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Step 6 (measurement).  Exact integer counters: vertices and kinks (each
   counted on its bond's lower site), worms, and the occupied imaginary time
   summed over sites (units beta/2^62, 128 bits).  Improved estimator of Q
   (Supplement S-I): on an interval of x = I eta between vertex legs (worms
   ignored) the worm density is eta tanh x (end states equal) or eta coth x
   (different), so sum_intervals x g(x) = beta eta <Q>.  A site without legs
   is one interval of x = beta eta with equal end states.                   */
static double xw_of(const or_handle* h) { return (h->p.beta * h->p.eta) * 0x1p-59; }

static void measure(or_handle* h, or_row* r) {
  memset(r, 0, sizeof *r);
  r->sweep = h->sweep;
  u128 occ = 0;
  double q = 0.0, XW = xw_of(h);
  for (int s = 0; s < h->N; s++) {
    const site_t* S = &h->site[s];
    int nl = 0;
    if (S->n == 0) { if (S->base) occ += (u128)TWO62; }
    for (int k = 0; k < S->n; k++) {
      uint64_t key = S->key[k];
      uint64_t nx = kpk(S->key[(k + 1) % S->n]);
      uint64_t len = (S->n == 1) ? TWO62 : ((nx - kpk(key)) & (TWO62 - 1));
      if (kab(key)) occ += (u128)len;
      if (kworm(key)) { r->n_w++; continue; }
      nl++;
      int a, d;
      leg_bond(h, s, ktag(key), &a, &d);
      if (a == s) { r->n_v++; if (kab(key) != kbl(key)) r->n_k++; }
    }
    if (ntau(h) > 1) {
      /* with temporal domains the estimator runs over the intervals of
         Step 4, delimited by the vertex legs and the temporal boundaries
         (whose states the configuration fixes), worms ignored */
      int NB = ntau(h), nd = nl + NB, j = 0;
      uint64_t* dl = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nd);
      for (int k = 0; k < S->n; k++) if (!kworm(S->key[k])) dl[j++] = S->key[k];
      for (int k = 0; k < NB; k++) {
        int b = state_at(S, tb_pk(h, k));
        dl[j++] = (tb_pk(h, k) << 2) | ((uint64_t)b << 1) | (uint64_t)b;
      }
      for (int i = 1; i < nd; i++)
        for (int m = i; m > 0 && kpk(dl[m]) < kpk(dl[m - 1]); m--) { uint64_t t = dl[m]; dl[m] = dl[m - 1]; dl[m - 1] = t; }
      for (int k = 0; k < nd; k++) {
        uint64_t lo = dl[k], hi = dl[(k + 1) % nd];
        double x = (double)wpts(kpk(lo), kpk(hi)) * XW;
        int sg = kab(lo) ^ kbl(hi);
        q = q + x * (sg ? coth_det(x) : tanh_det(x));
      }
      free(dl);
      continue;
    }
    if (nl == 0) { double x = (double)TWO59 * XW; q = q + x * tanh_det(x); continue; }
    int first = -1, prev = -1;
    for (int k = 0; k < S->n; k++) {
      if (kworm(S->key[k])) continue;
      if (first < 0) first = k;
      if (prev >= 0) {
        double x = (double)wpts(kpk(S->key[prev]), kpk(S->key[k])) * XW;
        int sg = kab(S->key[prev]) ^ kbl(S->key[k]);
        q = q + x * (sg ? coth_det(x) : tanh_det(x));
      }
      prev = k;
    }
    double x = (double)wpts(kpk(S->key[prev]), kpk(S->key[first])) * XW;
    int sg = kab(S->key[prev]) ^ kbl(S->key[first]);
    q = q + x * (sg ? coth_det(x) : tanh_det(x));
  }
  r->occ_lo = (uint64_t)occ;
  r->occ_hi = (uint64_t)(occ >> 64);
  r->q_impr = q;
  /* worms held by each domain (the paper's health figure of O(10)-O(100)
     worms per domain, discussion of Fig. 3): the fewest, and the empty ones */
  /* (a domain is a spatial domain times a temporal slab) */
  int nsd = h->ndom * ntau(h);
  uint64_t* wd = (uint64_t*)calloc((size_t)nsd, sizeof(uint64_t));
  for (int s = 0; s < h->N; s++)
    for (int k = 0; k < h->site[s].n; k++)
      if (kworm(h->site[s].key[k])) wd[dom_of(h, s) * ntau(h) + slab_of(h, kpk(h->site[s].key[k]))]++;
  uint64_t wmin = UINT64_MAX;
  for (int D = 0; D < nsd; D++) {
    if (wd[D] < wmin) wmin = wd[D];
    if (wd[D] == 0) r->dom_empty++;
  }
  r->w_dom_min = (uint32_t)wmin;
  free(wd);
}

static void push_row(or_handle* h, const or_row* r) {
  if (h->nrows == h->caprows) {
    h->caprows = h->caprows ? 2 * h->caprows : 1024;
    h->rows = (or_row*)realloc(h->rows, sizeof(or_row) * (size_t)h->caprows);
  }
  h->rows[h->nrows++] = *r;
}

/* ------------------------------------------------------------------------ */
/* Step 2 (spatial-boundary update, Eq. 4) on one boundary bond, then Step 3
   on that bond.  Its vertices are visited in time order.  For vertex v the
   four legs run to the next vertex leg on each site (worms ignored) with far
   states p (below) and q (above); if v is the only leg on a site, its two
   legs are one interval round the circle.  The new root states S' are drawn
   among the conserving ones with weight w(S') prod f_sigma(I eta), using
   f_0 = cosh, f_1 = sinh with the common factor e^x/2 dropped, i.e.
   f_sigma ~ 1 + (-1)^sigma e^{-2x} (computed from expm1_det).  Then the
   worms on the legs are drawn anew with the Eq. 1 sampler.                 */
typedef struct { int single; uint64_t plo, phi; int far_dn, far_up; uint64_t Idn, Iup, Ifull; } legs_t;

static void site_legs(const or_handle* h, int x, uint64_t pv, legs_t* L) {
  const site_t* S = &h->site[x];
  int iv = site_find(S, pv), n = S->n, jn = iv, jp = iv;
  for (int k = 0; k < n; k++) { jn = (jn + 1) % n; if (jn == iv || !kworm(S->key[jn])) break; }
  for (int k = 0; k < n; k++) { jp = (jp + n - 1) % n; if (jp == iv || !kworm(S->key[jp])) break; }
  L->single = (jn == iv);
  if (ntau(h) > 1) {
    /* with temporal domains a leg also ends at the nearest temporal
       boundary; its far state is the worldline's state there */
    uint64_t bu = tb_pk(h, tb_above(h, pv)), bd = tb_pk(h, tb_below(h, pv));
    if (L->single || up_dist(pv, bu) < up_dist(pv, kpk(S->key[jn]))) { L->phi = bu; L->far_up = state_at(S, bu); }
    else { L->phi = kpk(S->key[jn]); L->far_up = kbl(S->key[jn]); }
    if (L->single || up_dist(bd, pv) < up_dist(kpk(S->key[jp]), pv)) { L->plo = bd; L->far_dn = state_at(S, bd); }
    else { L->plo = kpk(S->key[jp]); L->far_dn = kab(S->key[jp]); }
    L->single = 0;
    L->Iup = wpts(pv, L->phi);
    L->Idn = wpts(L->plo, pv);
    return;
  }
  if (L->single) { L->Ifull = TWO59; L->plo = L->phi = pv; return; }
  L->phi = kpk(S->key[jn]); L->far_up = kbl(S->key[jn]); L->Iup = wpts(pv, L->phi);
  L->plo = kpk(S->key[jp]); L->far_dn = kab(S->key[jp]); L->Idn = wpts(L->plo, pv);
}

/* erase the worms strictly inside (lo, hi) going up (lo == hi: all), then
   draw new ones with p the state just above lo and q the state just below hi */
static int regen_interval(or_handle* h, stream_t* st, int x, uint64_t lo, uint64_t hi, int p, int q) {
  site_t* S = &h->site[x];
  uint64_t span = (hi > lo) ? hi - lo : hi + TWO62 - lo;
  for (int k = S->n - 1; k >= 0; k--) {
    if (!kworm(S->key[k])) continue;
    uint64_t off = (kpk(S->key[k]) + TWO62 - lo) & (TWO62 - 1);
    if (off > 0 && off < span) site_erase(S, k);
  }
  static uint64_t offs[MAXW];
  int n = sample_worms(&h->z, st, wpts(lo, hi), p ^ q, h->SWs, h->SWI, offs, MAXW);
  if (n < 0) return st->err ? st->err : OR_ETIMEOUT;
  uint64_t m0 = wm_above(lo);
  for (int k = 0; k < n; k++) site_add(S, wkey((m0 + offs[k]) & (TWO59 - 1), 0, p ^ 1 ^ (k & 1)), 0);
  fix_base(S);
  return OR_OK;
}

static double fsig(int sigma, double em1) { return sigma ? -em1 : 2.0 + em1; }

/* ------------------------------------------------------------------------ */
/* Step 1 (temporal-boundary update, Eq. 3) on one site.  Boundary k lies in
   the interval I = I2 + I1 between the nearest delimiters below and above it
   (vertex legs or other temporal boundaries, worms ignored): I2 from the lower
   delimiter (state p just above it) up to the boundary, I1 from the boundary
   up to the upper delimiter (state q just below it).  The new state s' at the
   boundary is drawn with P(s') = f_{q s'}(I1) f_{s' p}(I2) / f_{q p}(I), where
   f_{ab}(I) = <a| e^{I eta Q} |b> is cosh or sinh of x = I eta; written as
   e^x F(a ^ b, x) / 2 with F(0, x) = 2 + expm1(-2x), F(1, x) = -expm1(-2x),
   the factors e^x / 2 are common to both s' and drop out.  The worms of I2
   and I1 are then drawn anew with the Eq. 1 sampler (I2 first).  The
   boundaries of a site are updated one after the other, k = 0, 1, ..., each
   with the current states of the others (each update is a heat bath, so the
   sequence keeps the distribution); different sites are independent.      */
static void pdom_weights(int p, int q, uint64_t M1, uint64_t M2, double XW, double w[2]) {
  double e1 = or_expm1_det(-2.0 * ((double)M1 * XW)), e2 = or_expm1_det(-2.0 * ((double)M2 * XW));
  for (int sn = 0; sn < 2; sn++) w[sn] = fsig(q ^ sn, e1) * fsig(sn ^ p, e2);
}

void or_pdom(int p, int q, uint64_t M1, uint64_t M2, double XW, double out[2]) {
  double w[2];
  pdom_weights(p, q, M1, M2, XW, w);
  double tot = w[0] + w[1];
  out[0] = w[0] / tot;
  out[1] = w[1] / tot;
}

/* nearest delimiter of boundary point B going down (up = 0) or up (up = 1):
   its pk and the state on the side facing B */
static void tb_delim(const or_handle* h, const site_t* S, int k, int up, uint64_t* pk, int* st) {
  uint64_t B = tb_pk(h, k);
  int kb = up ? (k + 1) % ntau(h) : (k + ntau(h) - 1) % ntau(h);
  uint64_t best = tb_pk(h, kb);
  int from_leg = -1;
  for (int i = 0; i < S->n; i++) {
    if (kworm(S->key[i])) continue;
    uint64_t q = kpk(S->key[i]);
    if (up ? (up_dist(B, q) < up_dist(B, best)) : (up_dist(q, B) < up_dist(best, B))) { best = q; from_leg = i; }
  }
  *pk = best;
  if (from_leg >= 0) *st = up ? kbl(S->key[from_leg]) : kab(S->key[from_leg]);
  else *st = state_at(S, best);
}

static int step1_site(or_handle* h, int si) {
  site_t* S = &h->site[si];
  stream_t st;
  s_init(&st, h->p.seed, (uint32_t)si, c2_of(PH_TEMPORAL, 0, h->p.replica), (uint32_t)h->sweep);
  double XW = xw_of(h);
  for (int k = 0; k < ntau(h); k++) {
    uint64_t B = tb_pk(h, k), lo, hi;
    int p, q;
    tb_delim(h, S, k, 0, &lo, &p);
    tb_delim(h, S, k, 1, &hi, &q);
    double w[2];
    pdom_weights(p, q, wpts(B, hi), wpts(lo, B), XW, w);
    double tot = w[0] + w[1];
    if (!(tot > 0.0)) return OR_EINVARIANT;
    double u = ((double)(s_word(&st) >> 11) * 0x1p-53) * tot;
    int sn = (u < w[0]) ? 0 : 1;
    int rc = regen_interval(h, &st, si, lo, B, p, sn);
    if (rc == OR_OK) rc = regen_interval(h, &st, si, B, hi, sn, q);
    if (rc) return rc;
    if (S->n == 0) S->base = sn;
  }
  return st.err;
}

int or_temporal(or_handle* h) {
  if (ntau(h) < 2) return OR_OK;
  for (int s = 0; s < h->N; s++) {
    int rc = step1_site(h, s);
    if (rc) return rc;
  }
  return OR_OK;
}

static int step2_bond(or_handle* h, int a, int d) {
  int b = step(h, a, d, +1), tag = bond_tag(h, a, d);
  stream_t st;
  s_init(&st, h->p.seed, (uint32_t)(2 * a + d), c2_of(d ? PH_BY : PH_BX, 0, h->p.replica), (uint32_t)h->sweep);
  int nv = 0;
  const site_t* A = &h->site[a];
  uint64_t* pvs = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(A->n + 1));
  for (int k = 0; k < A->n; k++) if (ktag(A->key[k]) == tag) pvs[nv++] = kpk(A->key[k]);
  double XW = xw_of(h);
  int rc = OR_OK;
  for (int iv = 0; iv < nv && rc == OR_OK; iv++) {
    uint64_t pv = pvs[iv];
    legs_t La, Lb;
    site_legs(h, a, pv, &La);
    site_legs(h, b, pv, &Lb);
    double ea_dn = 0, ea_up, eb_dn = 0, eb_up;
    if (La.single) ea_up = or_expm1_det(-2.0 * ((double)La.Ifull * XW));
    else { ea_dn = or_expm1_det(-2.0 * ((double)La.Idn * XW)); ea_up = or_expm1_det(-2.0 * ((double)La.Iup * XW)); }
    if (Lb.single) eb_up = or_expm1_det(-2.0 * ((double)Lb.Ifull * XW));
    else { eb_dn = or_expm1_det(-2.0 * ((double)Lb.Idn * XW)); eb_up = or_expm1_det(-2.0 * ((double)Lb.Iup * XW)); }
    double cum[16], tot = 0.0;
    int lastS = -1;
    for (int S = 0; S < 16; S++) {
      double w = vweight(h, S);
      if (w > 0.0) {
        int s0 = S & 1, s1 = (S >> 1) & 1, s2 = (S >> 2) & 1, s3 = (S >> 3) & 1;
        if (!La.single) w = w * fsig(La.far_dn ^ s0, ea_dn);
        if (!Lb.single) w = w * fsig(Lb.far_dn ^ s1, eb_dn);
        w = w * (La.single ? fsig(s2 ^ s0, ea_up) : fsig(s2 ^ La.far_up, ea_up));
        w = w * (Lb.single ? fsig(s3 ^ s1, eb_up) : fsig(s3 ^ Lb.far_up, eb_up));
        if (w > 0.0) lastS = S;
      }
      tot = tot + w;
      cum[S] = tot;
    }
    if (lastS < 0) { rc = OR_EINVARIANT; break; }
    double u = ((double)(s_word(&st) >> 11) * 0x1p-53) * tot;
    int Sn = lastS;
    for (int S = 0; S < 16; S++) if (u < cum[S]) { Sn = S; break; }
    int s0 = Sn & 1, s1 = (Sn >> 1) & 1, s2 = (Sn >> 2) & 1, s3 = (Sn >> 3) & 1;
    site_t *SA = &h->site[a], *SB = &h->site[b];
    int ka = site_find(SA, pv), kb = site_find(SB, pv);
    SA->key[ka] = (SA->key[ka] & ~(uint64_t)3) | ((uint64_t)s0 << 1) | (uint64_t)s2;
    SB->key[kb] = (SB->key[kb] & ~(uint64_t)3) | ((uint64_t)s1 << 1) | (uint64_t)s3;
    fix_base(SA); fix_base(SB);
    if (!La.single) rc = regen_interval(h, &st, a, La.plo, pv, La.far_dn, s0);
    if (rc == OR_OK && !Lb.single) rc = regen_interval(h, &st, b, Lb.plo, pv, Lb.far_dn, s1);
    if (rc == OR_OK) rc = La.single ? regen_interval(h, &st, a, pv, pv, s2, s0)
                                    : regen_interval(h, &st, a, pv, La.phi, s2, La.far_up);
    if (rc == OR_OK) rc = Lb.single ? regen_interval(h, &st, b, pv, pv, s3, s1)
                                    : regen_interval(h, &st, b, pv, Lb.phi, s3, Lb.far_up);
  }
  free(pvs);
  if (rc == OR_OK && st.err) rc = st.err;
  if (rc == OR_OK) rc = step3_bond(h, a, d);
  return rc;
}

int or_boundary(or_handle* h) {
  for (int d = 0; d < 2; d++) {
    if ((d == 0 && h->ndx == 1) || (d == 1 && h->ndy == 1)) continue;
    for (int a = 0; a < h->N; a++) {
      if (!is_boundary_bond(h, a, d)) continue;
      int rc = step2_bond(h, a, d);
      if (rc) return rc;
    }
  }
  return OR_OK;
}

int or_tile(or_handle* h, int stop_after) {
  for (int a = 0; a < h->N; a++)
    for (int d = 0; d < 2; d++) {
      if (is_boundary_bond(h, a, d)) continue;
      int rc = step3_bond(h, a, d);
      if (rc) return rc;
    }
  if (stop_after <= 3) return OR_OK;
  for (int s = 0; s < h->N; s++) { int rc = step4_site(h, s); if (rc) return rc; }
  if (stop_after <= 4) return OR_OK;
  for (int p = 0; p < h->p.n_cycle; p++) { int rc = step5_pass(h, p); if (rc) return rc; }
  if (stop_after <= 5) return OR_OK;
  or_row r;
  measure(h, &r);
  push_row(h, &r);
  return OR_OK;
}

int or_sweep(or_handle* h, int64_t n) {
  for (int64_t k = 0; k < n; k++) {
    if ((h->ndx > 1 || h->ndy > 1 || ntau(h) > 1) && h->sweep % (uint64_t)h->K == 0) {
      int rc = or_temporal(h);                         /* Step 1 */
      if (rc == OR_OK && (h->ndx > 1 || h->ndy > 1)) rc = or_boundary(h);  /* Step 2 */
      if (rc) return rc;
    }
    int rc = or_tile(h, 6);
    if (rc) return rc;
    h->sweep++;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
static int validate(const or_params* p) {
  if (p->Lx < 2 || p->Ly < 2) return OR_EINVAL;
  if (!(p->beta > 0.0) || !(p->eta > 0.0) || !(p->t >= 0.0)) return OR_EINVAL;
  if (p->dom_x < 1 || p->dom_y < 1 || p->Lx % p->dom_x || p->Ly % p->dom_y) return OR_EINVAL;
  if (p->Lx / p->dom_x > 1 && p->dom_x < 2) return OR_EINVAL;
  if (p->Ly / p->dom_y > 1 && p->dom_y < 2) return OR_EINVAL;
  if (p->exchange_every < 1 || p->n_cycle < 0 || p->n_cycle > 4095) return OR_EINVAL;
  int B = p->sub_block;
  if (B < 0 || (B && (B & 1))) return OR_EINVAL;
  if (B && B < p->dom_x && p->dom_x % B) return OR_EINVAL;
  if (B && B < p->dom_y && p->dom_y % B) return OR_EINVAL;
  if (p->replica >= 65536 || p->init < 0 || p->init > 2) return OR_EINVAL;
  if (p->dom_tau < 1 || p->dom_tau > 64) return OR_EINVAL;
  if (!(p->vertex_window >= 0.0 && p->vertex_window <= 1.0)) return OR_EINVAL;
  /* the grid scales 2^59/(beta eta) and 2^59/(beta D) must lie in [2^39, 2^99] */
  if (!(p->beta * p->eta >= 0x1p-40 && p->beta * p->eta <= 0x1p20)) return OR_EINVAL;
  {
    or_handle t; memset(&t, 0, sizeof t); t.p = *p; derive(&t);
    if (t.D > 0.0 && !(p->beta * t.D >= 0x1p-40 && p->beta * t.D <= 0x1p20)) return OR_EINVAL;
  }
  return OR_OK;
}

int or_create(const or_params* p, or_handle** out) {
  int rc = validate(p);
  if (rc) return rc;
  or_handle* h = (or_handle*)calloc(1, sizeof(or_handle));
  h->p = *p;
  h->Lx = p->Lx; h->Ly = p->Ly; h->N = p->Lx * p->Ly;
  h->ndx = p->Lx / p->dom_x; h->ndy = p->Ly / p->dom_y; h->ndom = h->ndx * h->ndy;
  h->K = p->exchange_every;
  derive(h);
  zig_build(&h->z);
  h->site = (site_t*)calloc((size_t)h->N, sizeof(site_t));
  if (p->init == 1) {
    /* exactly floor(N/2) occupied sites: the first half of a Fisher-Yates
       permutation drawn from stream (init_seed, unit 0, init phase).       */
    int* perm = (int*)malloc(sizeof(int) * (size_t)h->N);
    for (int k = 0; k < h->N; k++) perm[k] = k;
    stream_t st;
    s_init(&st, p->init_seed, 0, c2_of(PH_INIT, 0, p->replica), 0);
    for (int k = h->N - 1; k >= 1; k--) {
      int j = (int)mulhi64(s_word(&st), (uint64_t)(k + 1));
      int t = perm[k]; perm[k] = perm[j]; perm[j] = t;
    }
    for (int k = 0; k < h->N / 2; k++) h->site[perm[k]].base = 1;
    free(perm);
  } else if (p->init == 2) {
    /* the checkerboard: site (x, y) occupied iff x + y is even */
    for (int s = 0; s < h->N; s++) h->site[s].base = ((sx(h, s) + sy(h, s)) & 1) == 0;
  }
  *out = h;
  return OR_OK;
}

void or_destroy(or_handle* h) {
  if (!h) return;
  for (int s = 0; s < h->N; s++) { free(h->site[s].key); free(h->site[s].lab); }
  free(h->site); free(h->rows); free(h);
}

int64_t or_rows(or_handle* h, or_row* out, int64_t max_rows) {
  int64_t n = h->nrows < max_rows ? h->nrows : max_rows;
  memcpy(out, h->rows, sizeof(or_row) * (size_t)n);
  memmove(h->rows, h->rows + n, sizeof(or_row) * (size_t)(h->nrows - n));
  h->nrows -= n;
  return n;
}

uint64_t or_sweep_index(or_handle* h) { return h->sweep; }
int or_set_sweep_index(or_handle* h, uint64_t s) { h->sweep = s; return OR_OK; }

size_t or_export_bytes(or_handle* h) {
  size_t n = 1 + (size_t)h->N;
  for (int s = 0; s < h->N; s++) n += (size_t)h->site[s].n;
  return n * sizeof(uint64_t);
}

int or_export(or_handle* h, void* buf, size_t bytes) {
  if (bytes < or_export_bytes(h)) return OR_EINVAL;
  uint64_t* o = (uint64_t*)buf;
  size_t k = 0;
  o[k++] = (uint64_t)h->N;
  for (int s = 0; s < h->N; s++) {
    const site_t* S = &h->site[s];
    o[k++] = (uint64_t)S->n | ((uint64_t)S->base << 63);
    for (int j = 0; j < S->n; j++) o[k++] = S->key[j];
  }
  return OR_OK;
}

int or_import(or_handle* h, const void* buf, size_t bytes) {
  const uint64_t* in = (const uint64_t*)buf;
  size_t nw = bytes / sizeof(uint64_t), k = 0;
  if (nw < 1 || in[0] != (uint64_t)h->N) return OR_EINVAL;
  k = 1;
  for (int s = 0; s < h->N; s++) {
    if (k >= nw) return OR_EINVAL;
    uint64_t hd = in[k++];
    int n = (int)(hd & 0x7fffffffu);
    if (k + (size_t)n > nw) return OR_EINVAL;
    site_t* S = &h->site[s];
    site_reserve(S, n);
    for (int j = 0; j < n; j++) { S->key[j] = in[k++]; S->lab[j] = 0; }
    S->n = n;
    S->base = (int)(hd >> 63);
  }
  return or_check(h);
}

/* Invariants of a configuration: keys strictly increasing in time; tags are
   bond legs (0..5) or worms (7); the state is continuous along every circle
   (state above an event = state below the next one, base = state above the
   last); every vertex leg has its partner leg at the same time on the other
   site of its bond; every vertex conserves particles, s0 + s1 = s2 + s3.   */
int or_check(or_handle* h) {
  for (int s = 0; s < h->N; s++) {
    const site_t* S = &h->site[s];
    for (int k = 0; k < S->n; k++) {
      uint64_t key = S->key[k];
      int t = ktag(key);
      if (t == 6) return OR_EINVARIANT;
      if (k > 0 && kpk(S->key[k - 1]) >= kpk(key)) return OR_EINVARIANT;
      if (kab(key) != kbl(S->key[(k + 1) % S->n])) return OR_EINVARIANT;
      if (t == 7) continue;
      int a, d;
      leg_bond(h, s, t, &a, &d);
      int b = step(h, a, d, +1);
      int other = (s == a) ? b : a;
      if (bond_tag(h, a, d) != t) return OR_EINVARIANT;
      int ko = site_find(&h->site[other], kpk(key));
      if (ko < 0) return OR_EINVARIANT;
      uint64_t ok = h->site[other].key[ko];
      uint64_t va = (s == a) ? key : ok, vb = (s == a) ? ok : key;
      if (kbl(va) + kbl(vb) != kab(va) + kab(vb)) return OR_EINVARIANT;
    }
    if (S->n && S->base != kab(S->key[S->n - 1])) return OR_EINVARIANT;
  }
  return OR_OK;
}

static double gfun(int sigma, double x) { return sigma ? coth_det(x) : tanh_det(x); }

/* ---- Supplement S-I resolved by the component of Q --------------------
   rho_a(X) = eta <q| e^{I2 eta Q} Q_a e^{I1 eta Q} |p> / <q| e^{I eta Q} |p>
   for X inside the interval I between two vertex legs of a site: p is the
   state above the lower leg, q the state below the upper one, I1 the part of
   I below X and I2 the part above.  For one site Q = b + b+ flips the state,
   so <a| e^{x Q} |b> = f_{ab}(x) = cosh x (a = b) or sinh x (a != b).
   Writing f_{ab}(x) = e^x F(a ^ b, x) / 2 with F(0, x) = 2 + expm1(-2x) and
   F(1, x) = -expm1(-2x), the factors e^x cancel because I1 + I2 = I (the
   lengths are counts of worm grid points, x = count * beta eta / 2^59):
     rho_a = eta F(q ^ out_a, I2) F(in_a ^ p, I1) / (2 F(q ^ p, I)),
   with Q_b taking 1 to 0 (in 1, out 0) and Q_b+ taking 0 to 1 (in 0, out 1).
   I1 counts the worm points strictly between the lower leg and X (0 when X
   sits on the leg), I2 = I - I1.
   A site without vertex legs is a circle with no reference point: the
   conditional density is the trace form eta Tr[Q_a e^{x Q}] / Tr[e^{x Q}]
   = eta F(1, x) / (2 F(0, x)) with x = beta eta (the whole circle).
   Two points on one interval (L below U going up from the lower leg, parts
   Ia, Ib, Ic from the bottom; the paper defers this case) follow from the
   same expansion with both operators inserted:
     eta^2 <q| e^{Ic Q} Q_U e^{Ib Q} Q_L e^{Ia Q} |p> / <q| e^{I Q} |p>
       = eta^2 F(q ^ out_U, Ic) F(in_U ^ out_L, Ib) F(in_L ^ p, Ia) / (4 F(q ^ p, I)),
   and on a site without legs (b+ ... going up from the point k1 to k2 over
   Ib points, the rest of the circle Ic = 2^59 - Ib):
     eta^2 Tr[Q_2 e^{Ib Q} Q_1 e^{Ic Q}] / Tr[e^{2^59 Q}]
       = eta^2 F(in_2 ^ out_1, Ib) F(in_1 ^ out_2, Ic) / (4 F(0, 2^59)).  */
static double Fsig(int sigma, uint64_t M, double XW) {
  double e = or_expm1_det(-2.0 * ((double)M * XW));
  return sigma ? -e : 2.0 + e;
}
static int q_in(int a) { return 1 - a; }   /* state below Q_a */
static int q_out(int a) { return a; }      /* state above Q_a */

typedef struct {
  int iv;          /* event index of the lower leg, -1: no legs */
  int p, q;        /* state above the lower leg, below the upper one */
  uint64_t M, M1;  /* worm points of the interval and below the slice */
  uint64_t off;    /* pk distance from the lower leg up to the slice */
  uint64_t pt;     /* the slice's pk */
} slice_t;

static uint64_t slice_pk(int32_t K, int k) { return (uint64_t)(((u128)k << 62) / (u128)K); }

static void slice_of(const site_t* S, uint64_t pt, slice_t* o) {
  o->pt = pt;
  int last = -1, lo = -1;
  for (int i = 0; i < S->n; i++)
    if (!kworm(S->key[i])) { last = i; if (kpk(S->key[i]) <= pt) lo = i; }
  if (last < 0) { o->iv = -1; o->p = o->q = 0; o->M = TWO59; o->M1 = 0; o->off = 0; return; }
  if (lo < 0) lo = last;                       /* the slice lies below the first leg */
  int hi = lo;                                 /* the next leg going up, cyclic */
  for (int i = 1; i <= S->n; i++) { hi = (lo + i) % S->n; if (!kworm(S->key[hi])) break; }
  uint64_t plo = kpk(S->key[lo]), phi = kpk(S->key[hi]);
  o->iv = lo;
  o->p = kab(S->key[lo]);
  o->q = kbl(S->key[hi]);
  o->M = wpts(plo, phi);
  o->M1 = (pt == plo) ? 0 : wpts(plo, pt);
  o->off = (pt - plo) & (TWO62 - 1);
}

static double rho_one(const slice_t* z, int a, double eta, double XW) {
  if (z->iv < 0) return eta * (Fsig(1, TWO59, XW) / (2.0 * Fsig(0, TWO59, XW)));
  double num = Fsig(z->q ^ q_out(a), z->M - z->M1, XW) * Fsig(q_in(a) ^ z->p, z->M1, XW);
  return eta * (num / (2.0 * Fsig(z->q ^ z->p, z->M, XW)));
}

/* Q_a1 at slice z1 and Q_a2 at slice z2, both on one interval of a site */
static double rho_two_same(const slice_t* z1, int a1, const slice_t* z2, int a2, double eta, double XW) {
  if (z1->iv < 0) {
    uint64_t Ib = wpts(z1->pt, z2->pt), Ic = TWO59 - Ib;
    double num = Fsig(q_in(a2) ^ q_out(a1), Ib, XW) * Fsig(q_in(a1) ^ q_out(a2), Ic, XW);
    return (eta * eta) * (num / (4.0 * Fsig(0, TWO59, XW)));
  }
  const slice_t *L = z1, *U = z2;
  int aL = a1, aU = a2;
  if (z2->off < z1->off) { L = z2; U = z1; aL = a2; aU = a1; }
  uint64_t Ia = L->M1, Ib = U->M1 - L->M1, Ic = L->M - U->M1;
  double num = (Fsig(L->q ^ q_out(aU), Ic, XW) * Fsig(q_in(aU) ^ q_out(aL), Ib, XW)) *
               Fsig(q_in(aL) ^ L->p, Ia, XW);
  return (eta * eta) * (num / (4.0 * Fsig(L->q ^ L->p, L->M, XW)));
}

int or_rho_alpha(or_handle* h, int32_t K, double* out, int32_t* iv) {
  if (K < 1) return OR_EINVAL;
  double XW = xw_of(h), eta = h->p.eta;
  for (int s = 0; s < h->N; s++)
    for (int k = 0; k < K; k++) {
      slice_t z;
      slice_of(&h->site[s], slice_pk(K, k), &z);
      size_t o = (size_t)s * (size_t)K + (size_t)k;
      for (int a = 0; a < 2; a++) out[o * 2 + (size_t)a] = rho_one(&z, a, eta, XW);
      if (iv) iv[o] = z.iv;
    }
  return OR_OK;
}

int or_rho_pair(or_handle* h, int32_t K, double* out) {
  if (K < 1) return OR_EINVAL;
  double XW = xw_of(h), eta = h->p.eta;
  slice_t* z = (slice_t*)malloc(sizeof(slice_t) * (size_t)K);
  for (int s = 0; s < h->N; s++) {
    for (int k = 0; k < K; k++) slice_of(&h->site[s], slice_pk(K, k), &z[k]);
    for (int k1 = 0; k1 < K; k1++)
      for (int k2 = 0; k2 < K; k2++)
        for (int a1 = 0; a1 < 2; a1++)
          for (int a2 = 0; a2 < 2; a2++) {
            double r;
            if (k1 == k2) r = 0.0;
            else if (z[k1].iv != z[k2].iv) r = rho_one(&z[k1], a1, eta, XW) * rho_one(&z[k2], a2, eta, XW);
            else r = rho_two_same(&z[k1], a1, &z[k2], a2, eta, XW);
            out[(((size_t)s * (size_t)K + (size_t)k1) * (size_t)K + (size_t)k2) * 4 + (size_t)(a1 * 2 + a2)] = r;
          }
  }
  free(z);
  return OR_OK;
}

/* n operators Q_a[0..g) at the points of one interval of a site, ordered in
   time going up from the interval's lower leg (Supplement S-I, with every
   operator inserted in the interval's matrix element; the paper leaves the
   case of several points on one interval to later work):
     eta^g <q| e^{I_g Q} Q_a[g-1] ... e^{I_1 Q} Q_a[0] e^{I_0 Q} |p> / <q| e^{I Q} |p>,
   where I_0 runs from the lower leg to the first point, I_j between points j-1
   and j, I_g from the last point to the upper leg (counts of worm points,
   M1[j] = the worm points strictly between the lower leg and point j).  Each
   Q_a maps its in-state to its out-state, so the states between the
   operators are fixed and the matrix element is the product of the factors
   f = e^x F / 2 of the pieces; the e^x cancel because the counts add up to I:
     eta^g F(q ^ out_a[g-1], I_g) ... F(in_a[j] ^ out_a[j-1], I_j) ... F(in_a[0] ^ p, I_0)
       / (2^g F(q ^ p, I)).
   p < 0 stands for a site without vertex legs: then the points lie on a circle
   with no reference point (M1[j] = the time point pk of point j, increasing),
   and the density is the cyclic trace
     eta^g Tr[e^{I_{g-1} Q} Q_a[g-1] ... e^{I_0 Q} Q_a[0]] / Tr[e^{2^59 Q}]
       = eta^g prod_j F(in_a[j+1] ^ out_a[j], I_j) / (2^g F(0, 2^59)),
   I_j the worm points strictly between points j and j + 1 for j < g - 1 and
   I_{g-1} = 2^59 minus their sum, the piece that closes the circle.        */
static double rho_interval(int p, int q, uint64_t M, int g, const uint64_t* M1, const int* a, double eta, double XW) {
  double num = 1.0, etag = 1.0;
  for (int j = 0; j < g; j++) etag = etag * eta;
  if (p < 0) {
    uint64_t used = 0;
    for (int j = 0; j < g; j++) {
      int nx = (j + 1) % g;
      uint64_t piece = (j + 1 < g) ? wpts(M1[j], M1[j + 1]) : TWO59 - used;
      used += piece;
      num = num * Fsig(q_in(a[nx]) ^ q_out(a[j]), piece, XW);
    }
    double den = 1.0;
    for (int j = 0; j < g; j++) den = den * 2.0;
    return etag * (num / (den * Fsig(0, TWO59, XW)));
  }
  num = Fsig(q_in(a[0]) ^ p, M1[0], XW);
  for (int j = 1; j < g; j++) num = num * Fsig(q_in(a[j]) ^ q_out(a[j - 1]), M1[j] - M1[j - 1], XW);
  num = num * Fsig(q ^ q_out(a[g - 1]), M - M1[g - 1], XW);
  double den = 1.0;
  for (int j = 0; j < g; j++) den = den * 2.0;
  return etag * (num / (den * Fsig(q ^ p, M, XW)));
}

double or_interval_density(int p, int q, uint64_t M, int g, const uint64_t* M1, const int* a, double eta, double XW) {
  return rho_interval(p, q, M, g, M1, a, eta, XW);
}

/* Supplement S-I n-point functions resolved by the component of Q at
   arbitrary times: for tuple j of n points (site s_c, slice k_c, component
   a_c) (pts[(j n + c) 3 + 0..2]), averaged over the K cyclic shifts t of all
   slices (tau_c = (k_c + t mod K) beta / K),
     out[j] = < Q_a1(X_1) ... Q_an(X_n) > = eta^-n < prod over intervals of the
              density of the points on that interval >,
   the points grouped by the interval (site and lower vertex leg, or the whole
   circle of a site without legs) that holds them, each group by the interval
   form above (a single point is rho_a of Supplement S-I), the groups
   multiplied in order of first appearance.  Two points of one tuple at the
   same site and slice are refused (OR_EINVAL).                              */
int or_npoint_alpha(or_handle* h, int32_t K, int32_t n, int64_t m, const int32_t* pts, double* out) {
  if (K < 1 || n < 1 || n > 16 || m < 0) return OR_EINVAL;
  double XW = xw_of(h), eta = h->p.eta;
  for (int64_t j = 0; j < m; j++) {
    const int32_t* t = pts + j * n * 3;
    for (int c = 0; c < n; c++) {
      if (t[3 * c] < 0 || t[3 * c] >= h->N || t[3 * c + 1] < 0 || t[3 * c + 1] >= K || (t[3 * c + 2] & ~1))
        return OR_EINVAL;
      for (int e = 0; e < c; e++)
        if (t[3 * e] == t[3 * c] && t[3 * e + 1] == t[3 * c + 1]) return OR_EINVAL;
    }
    double acc = 0.0;
    for (int sh = 0; sh < K; sh++) {
      slice_t z[16];
      for (int c = 0; c < n; c++) slice_of(&h->site[t[3 * c]], slice_pk(K, (t[3 * c + 1] + sh) % K), &z[c]);
      int done[16] = {0};
      double prod = 1.0;
      for (int c = 0; c < n; c++) {
        if (done[c]) continue;
        /* the points of c's interval, in time order going up from its lower
           leg (or from the circle's start on a site without legs) */
        int mem[16], g = 0;
        for (int e = c; e < n; e++)
          if (!done[e] && t[3 * e] == t[3 * c] && z[e].iv == z[c].iv) { mem[g++] = e; done[e] = 1; }
        for (int i = 1; i < g; i++)
          for (int k = i; k > 0; k--) {
            uint64_t ka = (z[c].iv < 0) ? z[mem[k]].pt : z[mem[k]].off;
            uint64_t kb = (z[c].iv < 0) ? z[mem[k - 1]].pt : z[mem[k - 1]].off;
            if (ka < kb) { int tmp = mem[k]; mem[k] = mem[k - 1]; mem[k - 1] = tmp; } else break;
          }
        uint64_t M1[16];
        int a[16];
        for (int i = 0; i < g; i++) {
          const slice_t* zi = &z[mem[i]];
          M1[i] = (z[c].iv < 0) ? zi->pt : zi->M1;
          a[i] = t[3 * mem[i] + 2];
        }
        prod = prod * rho_interval(z[c].iv < 0 ? -1 : z[c].p, z[c].q, z[c].M, g, M1, a, eta, XW);
      }
      acc = acc + prod;
    }
    double etan = 1.0;
    for (int c = 0; c < n; c++) etan = etan * eta;
    out[j] = (acc / (double)K) / etan;
  }
  return OR_OK;
}

int or_rho_slices(or_handle* h, int32_t K, double* out) {
  if (K < 1) return OR_EINVAL;
  double XW = xw_of(h), eta = h->p.eta;
  for (int s = 0; s < h->N; s++) {
    const site_t* S = &h->site[s];
    int nl = 0;
    for (int k = 0; k < S->n; k++) nl += !kworm(S->key[k]);
    uint64_t* lg = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nl + 1));
    nl = 0;
    for (int k = 0; k < S->n; k++) if (!kworm(S->key[k])) lg[nl++] = S->key[k];
    for (int k = 0; k < K; k++) {
      uint64_t pt = (uint64_t)(((u128)k << 62) / (u128)K);
      double r;
      if (nl == 0) { r = eta * tanh_det((double)TWO59 * XW); }
      else {
        int j = nl - 1;                     /* last leg with pk <= pt (cyclic) */
        for (int i = 0; i < nl; i++) if (kpk(lg[i]) <= pt) j = i;
        uint64_t lo = lg[j], hi = lg[(j + 1) % nl];
        double x = (double)wpts(kpk(lo), kpk(hi)) * XW;
        r = eta * gfun(kab(lo) ^ kbl(hi), x);
      }
      out[(size_t)s * (size_t)K + (size_t)k] = r;
    }
    free(lg);
  }
  return OR_OK;
}
