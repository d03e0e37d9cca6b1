// pmwa_kernels.cu -- sm_103a kernels of one PMWA Monte Carlo step.
//
//   k_boundary   Step 2 (Eq. 4) + Step 3 on the bonds between domains;
//                one warp per boundary bond, x bonds then y bonds, in
//                place on the current configuration.
//   k_rho        Supplement S-I worm density at equal-time slices.
//   k_check      invariants of the current configuration, one warp per site.
// Steps 3-6 of every other bond and site run in k_tile (pmwa_tile.cu).
//
// Configuration layout in HBM: site i owns the slot key[i*cap .. i*cap+cap)
// of 64-bit event keys sorted in time, and cnt[i] = count | base << 31.
#include <cuda_runtime.h>

#include <mutex>

#include "pmwa_device.cuh"

namespace pmwa {

static inline int blocks_for(long long n, int bs) { return int((n + bs - 1) / bs); }

constexpr int kMaxWormsPerInterval = 128;
constexpr uint32_t kCntMask = 0x7fffffffu;

__device__ __forceinline__ int cnt_n(uint32_t c) { return int(c & kCntMask); }
__device__ __forceinline__ int cnt_base(uint32_t c) { return int(c >> 31); }
__device__ __forceinline__ uint32_t cnt_make(int n, int base) { return uint32_t(n) | (uint32_t(base) << 31); }

// Supplement S-I worm density at K equal-time slices tau_k = k beta / K:
// eta g_sigma(x) of the interval between vertex legs holding tau_k.
__global__ void k_rho(const __grid_constant__ Dev d, int K, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.N) return;
  const uint64_t* Kk = d.keyA + size_t(s) * d.cap;
  const int n = cnt_n(d.cntA[s]);
  int nl = 0, lastleg = -1;
  for (int k = 0; k < n; ++k) if (!kworm(Kk[k])) { ++nl; lastleg = k; }
  const uint64_t q62 = kTwo62 / uint64_t(K), r62 = kTwo62 % uint64_t(K);
  for (int k = 0; k < K; ++k) {
    const uint64_t pt = uint64_t(k) * q62 + (uint64_t(k) * r62) / uint64_t(K);
    double r;
    if (nl == 0) {
      const double x = __dmul_rn(double(kTwo59), d.XW);
      r = __dmul_rn(d.eta, g_sigma(0, x));
    } else {
      int j = lastleg;   // last leg with pk <= pt, cyclic
      for (int i = 0; i < n; ++i) if (!kworm(Kk[i]) && kpk(Kk[i]) <= pt) j = i;
      int h = j;         // next leg after j, cyclic
      for (int i = 1; i <= n; ++i) { h = (j + i) % n; if (!kworm(Kk[h])) break; }
      const double x = __dmul_rn(__ull2double_rn(wpts(kpk(Kk[j]), kpk(Kk[h]))), d.XW);
      r = __dmul_rn(d.eta, g_sigma(kab(Kk[j]) ^ kbl(Kk[h]), x));
    }
    out[size_t(s) * K + k] = r;
  }
}

// ---------------------------------------------------------------------------
// Step 2 (spatial-boundary update, Eq. 4) and Step 3 on one boundary bond,
// in place on the current configuration.
__device__ __forceinline__ double vweight(const Dev& d, int S) {
  const int s0 = S & 1, s1 = (S >> 1) & 1, s2 = (S >> 2) & 1, s3 = (S >> 3) & 1;
  if (s0 + s1 != s2 + s3) return 0.0;
  if (s0 == s2) return d.dvw[s0 | (s1 << 1)];
  return d.tkink;
}

struct Legs {
  int single;
  uint64_t plo, phi, Idn, Iup;
  int far_dn, far_up;
  int wdn, wup;  // worms between the vertex and the next vertex leg below / above (0: none in the legs)
};

// the two legs of the vertex at pv on a site: to the next vertex leg below
// and above, worms ignored; one interval round the circle if v is alone.
// With temporal domains a leg also ends at the nearest temporal boundary,
// whose far state is the worldline's state there.
__device__ __noinline__ bool site_legs(const Dev& d, const uint64_t* K, int n, uint64_t pv, Legs* L) {
  const int iv = slot_find(K, n, pv);
  if (iv < 0) return false;
  int jn = iv, jp = iv, wu = 0, wd = 0;
  for (int k = 0; k < n; ++k) { jn = (jn + 1 == n) ? 0 : jn + 1; if (jn == iv || !kworm(K[jn])) break; ++wu; }
  for (int k = 0; k < n; ++k) { jp = (jp == 0) ? n - 1 : jp - 1; if (jp == iv || !kworm(K[jp])) break; ++wd; }
  L->single = (jn == iv);
  L->wup = wu;
  L->wdn = wd;
  if (d.ntau > 1) {
    const uint64_t bu = tb_pk(d, tb_above(d, pv)), bd = tb_pk(d, tb_below(d, pv));
    if (L->single || up_dist(pv, bu) < up_dist(pv, kpk(K[jn]))) { L->phi = bu; L->far_up = slot_state(K, n, 0, bu); }
    else { L->phi = kpk(K[jn]); L->far_up = kbl(K[jn]); }
    if (L->single || up_dist(bd, pv) < up_dist(kpk(K[jp]), pv)) { L->plo = bd; L->far_dn = slot_state(K, n, 0, bd); }
    else { L->plo = kpk(K[jp]); L->far_dn = kab(K[jp]); }
    L->single = 0;
    L->Iup = wpts(pv, L->phi);
    L->Idn = wpts(L->plo, pv);
    return true;
  }
  if (L->single) { L->plo = L->phi = pv; L->Idn = L->Iup = kTwo59; L->far_dn = L->far_up = 0; return true; }
  L->phi = kpk(K[jn]); L->far_up = kbl(K[jn]); L->Iup = wpts(pv, L->phi);
  L->plo = kpk(K[jp]); L->far_dn = kab(K[jp]); L->Idn = wpts(L->plo, pv);
  return true;
}

// Warp-cooperative list edits on a staged site list (all 32 lanes call them
// with the same arguments and see the same result).
//
// insert `key` at index `at`, shifting K[at..n) up by one, 32 keys at a time
// from the top (each chunk is read before any lane writes it)
__device__ __forceinline__ void aslot_insert(uint64_t* K, int n, int at, uint64_t key) {
  const int lane = threadIdx.x & 31;
  for (int top = n; top > at; top -= 32) {
    const int k = top - 1 - lane;
    const bool act = k >= at;
    uint64_t v = 0;
    if (act) v = K[k];
    __syncwarp();
    if (act) K[k + 1] = v;
    __syncwarp();
  }
  if (lane == 0) K[at] = key;
  __syncwarp();
}

// keep the keys for which drop(key) is false, in order; returns their count
template <class Drop>
__device__ __forceinline__ int warp_compact(uint64_t* K, int n, Drop drop) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int w = 0;
  for (int b = 0; b < n; b += 32) {
    const int k = b + lane;
    uint64_t key = 0;
    bool keep = false;
    if (k < n) { key = K[k]; keep = !drop(key); }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    __syncwarp();
    if (keep) K[w + __popc(m & lt)] = key;
    w += __popc(m);
    __syncwarp();
  }
  return w;
}

// first index >= from whose key has tag `tag` (n if none)
__device__ __forceinline__ int warp_find_tag(const uint64_t* K, int n, int from, int tag) {
  const int lane = threadIdx.x & 31;
  for (int b = from; b < n; b += 32) {
    const int k = b + lane;
    const unsigned m = __ballot_sync(0xffffffffu, k < n && ktag(K[k]) == tag);
    if (m) return b + __ffs(int(m)) - 1;
  }
  return n;
}

// erase the worms strictly inside (lo, hi) going up (lo == hi: all of them;
// erase false: the caller knows there are none) and draw new ones with end
// states p (above lo) and q (below hi); K holds n events (capacity cap).
__device__ __noinline__ int regen_interval(const Dev& d, const ZigTab& z, WarpStream& st, uint64_t* K, int& n,
                              uint64_t lo, uint64_t hi, int p, int q, bool erase) {
  const uint64_t span = (hi > lo) ? hi - lo : hi + kTwo62 - lo;
  if (erase)
    n = warp_compact(K, n, [&](uint64_t key) {  // the worms of the interval
      if (!kworm(key)) return false;
      const uint64_t off = (kpk(key) + kTwo62 - lo) & (kTwo62 - 1);
      return off > 0 && off < span;
    });
  uint64_t offs[kMaxWormsPerInterval];
  int bad = 0;
  const int nw = sample_worms<kMaxWormsPerInterval>(z, st, wpts(lo, hi), p ^ q, d.SWs, d.SWI, offs, &bad);
  if (bad) return bad;
  const uint64_t m0 = wm_above(lo);
  for (int k = 0; k < nw; ++k) {
    if (n >= d.cap) return PMWA_ECAPACITY;
    const uint64_t key = wkey((m0 + offs[k]) & (kTwo59 - 1), 0, p ^ 1 ^ (k & 1));
    aslot_insert(K, n, slot_lower(K, n, kpk(key)), key);
    ++n;
  }
  return PMWA_OK;
}

__device__ __forceinline__ double fsig(int sigma, double em1) { return sigma ? -em1 : __dadd_rn(2.0, em1); }

// Eq. 4 in binary32 (lane < 16: state S = lane; all 32 lanes call it): the
// same heat bath with the leg factors from expm1f and the vertex weights
// rounded to binary32.  Its cumulative fractions c_S / tot lie within 2^-16
// of the binary64 ones (expm1f within a few units in the last place, at
// most four factors and one vertex weight, a sum of at most six terms, each
// a relative 2^-22 or better), so when the uniform r = (w >> 11) 2^-53 lies
// more than 2^-12 from 0, 1 and every boundary, the binary64 computation
// picks the same state.  (A state whose binary32 weight vanishes while its
// binary64 one does not has a fraction below 2^-100 and so sits within the
// margin of a neighbouring boundary or of 0.)  Returns that state, or -1.
__device__ int heat_bath_f32(const Dev& d, const Legs& La, const Legs& Lb, uint64_t w, int lane) {
  float e4 = 0.f;
  if (lane < 4) {
    uint64_t I;
    if (lane == 0) I = La.single ? kTwo59 : La.Idn;
    else if (lane == 1) I = Lb.single ? kTwo59 : Lb.Idn;
    else if (lane == 2) I = La.single ? kTwo59 : La.Iup;
    else I = Lb.single ? kTwo59 : Lb.Iup;
    e4 = expm1f(-2.0f * __ull2float_rn(I) * d.XWf);
  }
  const float ea_dn = __shfl_sync(0xffffffffu, e4, 0), eb_dn = __shfl_sync(0xffffffffu, e4, 1);
  const float ea_up = __shfl_sync(0xffffffffu, e4, 2), eb_up = __shfl_sync(0xffffffffu, e4, 3);
  float wS = 0.f;
  if (lane < 16) {
    const int S = lane, s0 = S & 1, s1 = (S >> 1) & 1, s2 = (S >> 2) & 1, s3 = (S >> 3) & 1;
    if (s0 + s1 == s2 + s3) {
      float v = (s0 == s2) ? d.dvwf[s0 | (s1 << 1)] : d.tkinkf;
      auto f = [](int sg, float e) { return sg ? -e : 2.0f + e; };
      if (!La.single) v *= f(La.far_dn ^ s0, ea_dn);
      if (!Lb.single) v *= f(Lb.far_dn ^ s1, eb_dn);
      v *= La.single ? f(s2 ^ s0, ea_up) : f(s2 ^ La.far_up, ea_up);
      v *= Lb.single ? f(s3 ^ s1, eb_up) : f(s3 ^ Lb.far_up, eb_up);
      wS = v;
    }
  }
  float c = wS;  // inclusive running sums over the states
  for (int o = 1; o < 16; o <<= 1) {
    const float t = __shfl_up_sync(0xffffffffu, c, o);
    if (lane >= o) c += t;
  }
  const float tot = __shfl_sync(0xffffffffu, c, 15);
  if (!(tot > 0x1p-100f)) return -1;
  const float r = __ull2float_rn(w >> 11) * 0x1p-53f;
  const float fr = c / tot;
  const bool pos = lane < 16 && wS > 0.f;
  const bool near = (pos && fabsf(r - fr) <= 0x1p-12f) || r <= 0x1p-12f;
  if (__any_sync(0xffffffffu, near)) return -1;
  const unsigned hit = __ballot_sync(0xffffffffu, pos && r < fr);
  return hit ? __ffs(int(hit)) - 1 : -1;
}
__device__ __forceinline__ double em1_of(uint64_t I, double XW) {
  return expm1_det(__dmul_rn(-2.0, __dmul_rn(__ull2double_rn(I), XW)));
}

__device__ __forceinline__ int boundary_count(const Dev& d, int dir) {
  return dir == 0 ? (d.ndx > 1 ? d.ndx * d.Ly : 0) : (d.ndy > 1 ? d.ndy * d.Lx : 0);
}

// lower site of boundary bond number t of direction dir
__device__ __forceinline__ int boundary_site(const Dev& d, int dir, int t) {
  if (dir == 0) return ((t % d.ndx) * d.dom_x + d.dom_x - 1) + d.Lx * (t / d.ndx);
  return (t % d.Lx) + d.Lx * ((t / d.Lx) * d.dom_y + d.dom_y - 1);
}

// On-the-fly vertex generation: is grid point pos within half of a worm of
// either staged list (cyclic)?
__device__ __forceinline__ bool in_win_lists(const uint64_t* KA, int nA, const uint64_t* KB, int nB, uint64_t pos,
                                             uint64_t half) {
  for (int side = 0; side < 2; ++side) {
    const uint64_t* K = side ? KB : KA;
    const int n = side ? nB : nA;
    for (int i = 0; i < n; ++i) {
      if (!kworm(K[i])) continue;
      const uint64_t m = kpk(K[i]) >> 3;
      const uint64_t a = (pos - m) & (kTwo59 - 1), b = (m - pos) & (kTwo59 - 1);
      if (min(a, b) <= half) return true;
    }
  }
  return false;
}

// Step 2 + Step 3 on the boundary bond (a, dir) whose two site lists are
// staged in KA (nA events) and KB (nB events); returns a status.  With
// d.win_half > 0 the Step-3 part is confined to the windows around the worms
// of the two sites (on-the-fly vertex generation).
__device__ int boundary_bond_update(const Dev& d, int a, int dir, uint64_t* KA, int& nA, int& baseA,
                                    uint64_t* KB, int& nB, int& baseB, const ZigTab& Z) {
  const int tag = bond_tag(d, a, dir);
  const int bid = 2 * a + dir;
  WarpStream st;
  st.init(d.key0, d.key1, uint32_t(bid), c2_word(dir ? kBy : kBx, 0, d.replica), d.sweep);
  int rc = PMWA_OK;
  // Step 2: the bond's vertices in time order (worms move, vertices do not)
  uint64_t last = 0;
  bool any = false;
  for (;;) {
    const int k = warp_find_tag(KA, nA, any ? slot_lower(KA, nA, last + 1) : 0, tag);
    if (k >= nA) break;
    const uint64_t pv = kpk(KA[k]);
    last = pv;
    any = true;
    Legs La, Lb;
    if (!site_legs(d, KA, nA, pv, &La) || !site_legs(d, KB, nB, pv, &Lb)) return PMWA_EINVARIANT;
    // heat-bath over the root states (Eq. 4): decided in binary32 when the
    // uniform lies clear of every boundary, else in binary64 with one lane
    // per leg factor and one lane per state and the weights summed in the
    // fixed order S = 0..15
    const int lane = threadIdx.x & 31;
    const uint64_t wu = st.word();
    int Sn = heat_bath_f32(d, La, Lb, wu, lane);
    if (Sn < 0) {
    double e4 = 0.0;
    if (lane < 4) {
      uint64_t I;
      if (lane == 0) I = La.single ? kTwo59 : La.Idn;
      else if (lane == 1) I = Lb.single ? kTwo59 : Lb.Idn;
      else if (lane == 2) I = La.single ? kTwo59 : La.Iup;
      else I = Lb.single ? kTwo59 : Lb.Iup;
      e4 = em1_of(I, d.XW);
    }
    const double ea_dn = __shfl_sync(0xffffffffu, e4, 0), eb_dn = __shfl_sync(0xffffffffu, e4, 1);
    const double ea_up = __shfl_sync(0xffffffffu, e4, 2), eb_up = __shfl_sync(0xffffffffu, e4, 3);
    double wS = 0.0;
    if (lane < 16) {
      const int S = lane;
      double w = vweight(d, S);
      if (w > 0.0) {
        const int s0 = S & 1, s1 = (S >> 1) & 1, s2 = (S >> 2) & 1, s3 = (S >> 3) & 1;
        if (!La.single) w = __dmul_rn(w, fsig(La.far_dn ^ s0, ea_dn));
        if (!Lb.single) w = __dmul_rn(w, fsig(Lb.far_dn ^ s1, eb_dn));
        w = __dmul_rn(w, La.single ? fsig(s2 ^ s0, ea_up) : fsig(s2 ^ La.far_up, ea_up));
        w = __dmul_rn(w, Lb.single ? fsig(s3 ^ s1, eb_up) : fsig(s3 ^ Lb.far_up, eb_up));
      }
      wS = w;
    }
    // running sums in the order S = 0..15 over the states of non-zero
    // weight only (adding +0.0 changes no sum, so this is the sequential
    // sum over all 16); a zero-weight state keeps cumS = 0 and is never hit
    const unsigned pos = __ballot_sync(0xffffffffu, lane < 16 && wS > 0.0);
    if (!pos) return PMWA_EINVARIANT;
    double tot = 0.0, cumS = 0.0;
    for (unsigned m = pos; m; m &= m - 1) {
      const int S = __ffs(int(m)) - 1;
      tot = __dadd_rn(tot, __shfl_sync(0xffffffffu, wS, S));
      if (lane == S) cumS = tot;
    }
    const int lastS = 31 - __clz(int(pos));
    const double u = __dmul_rn(__dmul_rn(__ull2double_rn(wu >> 11), 0x1p-53), tot);
    const unsigned hit = __ballot_sync(0xffffffffu, lane < 16 && u < cumS);
    Sn = hit ? (__ffs(int(hit)) - 1) : lastS;
    }
    const int s0 = Sn & 1, s1 = (Sn >> 1) & 1, s2 = (Sn >> 2) & 1, s3 = (Sn >> 3) & 1;
    {
      const int ka = slot_find(KA, nA, pv), kb = slot_find(KB, nB, pv);
      if (ka < 0 || kb < 0) return PMWA_EINVARIANT;
      KA[ka] = (KA[ka] & ~3ull) | (uint64_t(s0) << 1) | uint64_t(s2);
      KB[kb] = (KB[kb] & ~3ull) | (uint64_t(s1) << 1) | uint64_t(s3);
    }
    // (the worm counts of the legs were taken before any redraw; a redraw
    // below v adds worms only below v, so the counts above v still hold)
    if (!La.single) rc = regen_interval(d, Z, st, KA, nA, La.plo, pv, La.far_dn, s0, La.wdn > 0);
    if (!rc && !Lb.single) rc = regen_interval(d, Z, st, KB, nB, Lb.plo, pv, Lb.far_dn, s1, Lb.wdn > 0);
    if (!rc) rc = La.single ? regen_interval(d, Z, st, KA, nA, pv, pv, s2, s0, La.wup > 0)
                            : regen_interval(d, Z, st, KA, nA, pv, La.phi, s2, La.far_up, La.wup > 0);
    if (!rc) rc = Lb.single ? regen_interval(d, Z, st, KB, nB, pv, pv, s3, s1, Lb.wup > 0)
                            : regen_interval(d, Z, st, KB, nB, pv, Lb.phi, s3, Lb.far_up, Lb.wup > 0);
    if (rc) return rc;
  }
  if (st.pos >= (uint64_t(1) << 33)) return PMWA_ETIMEOUT;
  // states at the start of the circles after Step 2 (used if a list empties)
  if (nA) baseA = kab(KA[nA - 1]);
  if (nB) baseB = kab(KB[nB - 1]);
  // Step 3 on this bond: erase its diagonal vertices, lay new ones
  const bool otf = d.win_half > 0;
  {
    // (the windows do not move: the compaction drops only diagonal legs, so
    // while it runs every worm of both lists is still found in their first
    // nA / nB slots, some of them twice, which the window test does not mind)
    auto diag = [&](uint64_t key) {
      return ktag(key) == tag && kab(key) == kbl(key) &&
             (!otf || in_win_lists(KA, nA, KB, nB, kpk(key) >> 3, d.win_half));
    };
    const int wa = warp_compact(KA, nA, diag);
    const int wb = warp_compact(KB, nB, diag);
    const int removed = nA - wa, gone = nB - wb;
    nA = wa;
    nB = wb;
    if (gone != removed) return PMWA_EINVARIANT;
  }
  if (!d.has_vertices) return PMWA_OK;
  WarpStream sv;
  sv.init(d.key0, d.key1, uint32_t(bid), c2_word(kVertex, 0, d.replica), d.sweep);
  uint64_t pos = 0;
  bool first = true;
  int bad = 0;
  for (;;) {
    const uint64_t E = zig_exp(Z, sv, &bad);
    if (bad) return bad;
    const uint64_t g = grid_gap(E, d.SVs);
    const uint64_t nxt = first ? g - 1 : pos + g;
    first = false;
    if (nxt >= kTwo59) break;
    pos = nxt;
    const uint64_t pk = (pos << 3) | uint64_t(tag);
    if (otf && !in_win_lists(KA, nA, KB, nB, pos, d.win_half)) continue;
    if (slot_find(KA, nA, pk) >= 0) continue;
    const int na = slot_state(KA, nA, baseA, pk), nb = slot_state(KB, nB, baseB, pk);
    const int si = na | (nb << 1);
    if (d.TV[si] < kTwo32) {
      const uint64_t w = sv.word();
      if ((w >> 32) >= d.TV[si]) continue;
    }
    if (nA >= d.cap || nB >= d.cap) return PMWA_ECAPACITY;
    aslot_insert(KA, nA, slot_lower(KA, nA, pk), (pk << 2) | (uint64_t(na) << 1) | uint64_t(na));
    ++nA;
    aslot_insert(KB, nB, slot_lower(KB, nB, pk), (pk << 2) | (uint64_t(nb) << 1) | uint64_t(nb));
    ++nB;
  }
  return PMWA_OK;
}

// One warp per boundary bond.  The warp copies the bond's two site lists
// into its shared-memory stage (coalesced), every lane then runs the same
// update on the same data (so nothing diverges; lanes split only the
// heat-bath arithmetic), and the warp copies the lists back.  stage: 2 * cap
// event keys for this warp.
__device__ void boundary_warp(const Dev& d, int dir, int t, uint64_t* stage, const ZigTab& Z) {
  const int lane = threadIdx.x & 31;
  if (t >= boundary_count(d, dir)) return;
  const int a = boundary_site(d, dir, t);
  const int b = site_step(d, a, dir, +1);
  const uint32_t ca = d.cntA[a], cb = d.cntA[b];
  int nA = cnt_n(ca), baseA = cnt_base(ca), nB = cnt_n(cb), baseB = cnt_base(cb);
  const uint64_t* ga = d.keyA + size_t(a) * d.cap;
  const uint64_t* gb = d.keyA + size_t(b) * d.cap;
  uint64_t* sa = stage;
  uint64_t* sb = stage + d.cap;
  for (int k = lane; k < nA; k += 32) sa[k] = ga[k];
  for (int k = lane; k < nB; k += 32) sb[k] = gb[k];
  __syncwarp();
  const int rc = boundary_bond_update(d, a, dir, sa, nA, baseA, sb, nB, baseB, Z);
  __syncwarp();
  if (rc) {
    if (lane == 0) set_err(d.err, rc, 2);
    return;
  }
  uint64_t* wa = d.keyA + size_t(a) * d.cap;
  uint64_t* wb = d.keyA + size_t(b) * d.cap;
  for (int k = lane; k < nA; k += 32) wa[k] = sa[k];
  for (int k = lane; k < nB; k += 32) wb[k] = sb[k];
  if (lane == 0) {
    d.cntA[a] = cnt_make(nA, nA ? kab(sa[nA - 1]) : baseA);
    d.cntA[b] = cnt_make(nB, nB ? kab(sb[nB - 1]) : baseB);
  }
}

constexpr int kBoundaryWarps = 4;  // bonds (warps) per block

__global__ void __launch_bounds__(32 * kBoundaryWarps) k_boundary(const __grid_constant__ Dev d, int dir) {
  extern __shared__ __align__(16) unsigned char bsm[];
  if (instance_failed(d.err)) return;
  const ZigTab Z = zig_stage(bsm, d.zig_cap, d.worm_tries);
  __syncthreads();
  const int wid = threadIdx.x >> 5;
  uint64_t* stage = reinterpret_cast<uint64_t*>(bsm + kZigBytes) + size_t(2 * wid) * d.cap;
  boundary_warp(d, dir, int(blockIdx.x) * kBoundaryWarps + wid, stage, Z);
}

// Batched form: each block serves bonds t0 .. t0 + kBoundaryWarps - 1 of one
// instance, when that instance's boundary step is due at iteration `it`.
__global__ void __launch_bounds__(32 * kBoundaryWarps) k_boundary_batch(const Dev* __restrict__ devs,
                                                                        const BatchBase* __restrict__ base,
                                                                        const int2* __restrict__ work, int it,
                                                                        int dir, int cap) {
  extern __shared__ __align__(16) unsigned char bsm[];
  __shared__ Dev sd;
  const int2 w = work[blockIdx.x];
  const BatchBase bb = base[w.x];
  if (!bb.active) return;
  if (threadIdx.x == 0) sd = at_iteration(devs[w.x], bb, it);
  ZigTab Z = zig_stage(bsm);
  __syncthreads();
  Z.zcap = sd.zig_cap;
  Z.wtries = sd.worm_tries;
  if (instance_failed(sd.err)) return;
  if (sd.ndom < 2 || sd.sweep % uint32_t(sd.exchange_every) != 0) return;
  const int wid = threadIdx.x >> 5;
  uint64_t* stage = reinterpret_cast<uint64_t*>(bsm + kZigBytes) + size_t(2 * wid) * cap;
  boundary_warp(sd, dir, w.y + wid, stage, Z);
}

// ---------------------------------------------------------------------------
// Step 1 (temporal-boundary update, Eq. 3), one warp per site, in place on
// the current configuration.  Boundary k lies in the interval I = I2 + I1
// between the nearest delimiters below and above it (vertex legs or other
// temporal boundaries, worms ignored): I2 from the lower delimiter (state p
// just above it) up to the boundary, I1 from the boundary up to the upper one
// (state q just below it).  The new state s' is drawn with P(s') =
// f_{q s'}(I1) f_{s' p}(I2) / f_{q p}(I); with f_{ab}(x) = e^x F(a ^ b, x) / 2,
// F(0, x) = 2 + expm1(-2x), F(1, x) = -expm1(-2x), the e^x / 2 are common to
// both s' and drop out.  The worms of I2 and then I1 are drawn anew (Eq. 1).
// The boundaries of a site go in order k = 0, 1, ..., each a heat bath given
// the current states of the others; sites are independent.  Every lane runs
// the same update on the staged list, as in the spatial boundary step.

// the nearest delimiter of boundary k going down (up = false) or up: its pk
// and the state on the side facing the boundary
__device__ __forceinline__ void tb_delim(const Dev& d, const uint64_t* K, int n, int base, int k, bool up,
                                         uint64_t* pk, int* st) {
  const uint64_t B = tb_pk(d, k);
  const int kb = up ? (k + 1) % d.ntau : (k + d.ntau - 1) % d.ntau;
  uint64_t best = tb_pk(d, kb);
  int leg = -1;
  if (n > 0) {
    // the nearest vertex leg in that direction, cyclic (worms skipped)
    const int i0 = slot_lower(K, n, B);  // first event above B
    for (int c = 0; c < n; ++c) {
      const int i = up ? (i0 + c) % n : (i0 + n - 1 - c) % n;
      if (kworm(K[i])) continue;
      const uint64_t q = kpk(K[i]);
      if (up ? up_dist(B, q) < up_dist(B, best) : up_dist(q, B) < up_dist(best, B)) { best = q; leg = i; }
      break;
    }
  }
  *pk = best;
  *st = (leg >= 0) ? (up ? kbl(K[leg]) : kab(K[leg])) : slot_state(K, n, base, best);
}

__device__ int temporal_site(const Dev& d, int s, uint64_t* K, int& n, int& base, const ZigTab& Z) {
  WarpStream st;
  st.init(d.key0, d.key1, uint32_t(s), c2_word(kTemporal, 0, d.replica), d.sweep);
  for (int k = 0; k < d.ntau; ++k) {
    const uint64_t B = tb_pk(d, k);
    uint64_t lo, hi;
    int p, q;
    tb_delim(d, K, n, base, k, false, &lo, &p);
    tb_delim(d, K, n, base, k, true, &hi, &q);
    const uint64_t I1 = wpts(B, hi), I2 = wpts(lo, B);
    const uint64_t wu = st.word();
    // decided in binary32 when the uniform lies more than 2^-12 from the
    // fraction w0 / (w0 + w1) (two leg factors: the binary32 fraction is
    // within 2^-18 of the binary64 one), else in binary64
    int sn;
    {
      auto f = [](int sg, float e) { return sg ? -e : 2.0f + e; };
      const float g1 = expm1f(-2.0f * __ull2float_rn(I1) * d.XWf), g2 = expm1f(-2.0f * __ull2float_rn(I2) * d.XWf);
      const float v0 = f(q, g1) * f(p, g2), v1 = f(q ^ 1, g1) * f(1 ^ p, g2);
      const float r = __ull2float_rn(wu >> 11) * 0x1p-53f, fr = v0 / (v0 + v1);
      sn = (v0 + v1 > 0x1p-100f && fabsf(r - fr) > 0x1p-12f && r > 0x1p-12f) ? (r < fr ? 0 : 1) : -1;
    }
    if (sn < 0) {
      const double e1 = em1_of(I1, d.XW), e2 = em1_of(I2, d.XW);
      const double w0 = __dmul_rn(fsig(q, e1), fsig(p, e2));
      const double w1 = __dmul_rn(fsig(q ^ 1, e1), fsig(1 ^ p, e2));
      const double tot = __dadd_rn(w0, w1);
      if (!(tot > 0.0)) return PMWA_EINVARIANT;
      const double u = __dmul_rn(__dmul_rn(__ull2double_rn(wu >> 11), 0x1p-53), tot);
      sn = (u < w0) ? 0 : 1;
    }
    int rc = regen_interval(d, Z, st, K, n, lo, B, p, sn, true);
    if (!rc) rc = regen_interval(d, Z, st, K, n, B, hi, sn, q, true);
    if (rc) return rc;
    if (n == 0) base = sn;
  }
  if (st.pos >= (uint64_t(1) << 33)) return PMWA_ETIMEOUT;
  return PMWA_OK;
}

constexpr int kTemporalWarps = 4;  // sites (warps) per block

// one warp: stage site s's list (cap keys at K), update its boundaries, and
// write it back
__device__ void temporal_warp(const Dev& d, int s, uint64_t* K, const ZigTab& Z) {
  const int lane = threadIdx.x & 31;
  if (s >= d.N) return;
  const uint32_t c = d.cntA[s];
  int n = cnt_n(c), base = cnt_base(c);
  const uint64_t* g = d.keyA + size_t(s) * d.cap;
  for (int k = lane; k < n; k += 32) K[k] = g[k];
  __syncwarp();
  const int rc = temporal_site(d, s, K, n, base, Z);
  __syncwarp();
  if (rc) {
    if (lane == 0) set_err(d.err, rc, 1);
    return;
  }
  uint64_t* w = d.keyA + size_t(s) * d.cap;
  for (int k = lane; k < n; k += 32) w[k] = K[k];
  if (lane == 0) d.cntA[s] = cnt_make(n, n ? kab(K[n - 1]) : base);
}

__global__ void __launch_bounds__(32 * kTemporalWarps) k_temporal(const __grid_constant__ Dev d) {
  extern __shared__ __align__(16) unsigned char tsm[];
  if (instance_failed(d.err)) return;
  const ZigTab Z = zig_stage(tsm, d.zig_cap, d.worm_tries);
  __syncthreads();
  const int wid = threadIdx.x >> 5;
  temporal_warp(d, int(blockIdx.x) * kTemporalWarps + wid,
                reinterpret_cast<uint64_t*>(tsm + kZigBytes) + size_t(wid) * d.cap, Z);
}

// Batched form: each block serves sites t0 .. t0 + kTemporalWarps - 1 of one
// instance, when that instance has temporal domains and its Step 1 is due at
// iteration `it`.
__global__ void __launch_bounds__(32 * kTemporalWarps) k_temporal_batch(const Dev* __restrict__ devs,
                                                                        const BatchBase* __restrict__ base,
                                                                        const int2* __restrict__ work, int it,
                                                                        int cap) {
  extern __shared__ __align__(16) unsigned char tsm[];
  __shared__ Dev sd;
  const int2 w = work[blockIdx.x];
  const BatchBase bb = base[w.x];
  if (!bb.active) return;
  if (threadIdx.x == 0) sd = at_iteration(devs[w.x], bb, it);
  ZigTab Z = zig_stage(tsm);
  __syncthreads();
  Z.zcap = sd.zig_cap;
  Z.wtries = sd.worm_tries;
  if (instance_failed(sd.err)) return;
  if (sd.ntau < 2 || sd.sweep % uint32_t(sd.exchange_every) != 0) return;
  const int wid = threadIdx.x >> 5;
  temporal_warp(sd, w.y + wid, reinterpret_cast<uint64_t*>(tsm + kZigBytes) + size_t(wid) * cap, Z);
}

static size_t temporal_smem(int cap) { return size_t(kZigBytes) + size_t(kTemporalWarps) * size_t(cap) * 8; }

int temporal_sites_per_block() { return kTemporalWarps; }

int launch_temporal(const Dev& d, void* stream) {
  if (d.ntau < 2) return 0;
  const size_t smem = temporal_smem(d.cap);
  cudaError_t e = cudaFuncSetAttribute(k_temporal, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e) return int(e);
  k_temporal<<<blocks_for(d.N, kTemporalWarps), 32 * kTemporalWarps, smem, cudaStream_t(stream)>>>(d);
  return int(cudaGetLastError());
}

// (the batch sets the kernel's shared-memory allowance once, before any
// capture: prepare_temporal)
int prepare_temporal(int cap) {
  return int(cudaFuncSetAttribute(k_temporal_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(temporal_smem(cap))));
}

int launch_temporal_batch(const Dev* devs, const BatchBase* base, const int2* work, int n_work, int it, int cap,
                          void* stream) {
  if (n_work <= 0) return 0;
  k_temporal_batch<<<n_work, 32 * kTemporalWarps, temporal_smem(cap), cudaStream_t(stream)>>>(devs, base, work, it,
                                                                                              cap);
  return int(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Launchers.

int upload_zig(const Zig& z) { return upload_constants(z); }

// advance every instance's batch state by S sweeps (the tail of a captured
// sequence of S sweeps, so that the next replay continues where it ended)
__global__ void k_advance(BatchBase* base, int n, int S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !base[i].active) return;
  base[i].sweep0 += uint32_t(S);
  base[i].row0 += S;
  base[i].flip ^= (S & 1);
}

int launch_advance(BatchBase* base, int n, int S, void* stream) {
  k_advance<<<blocks_for(n, 128), 128, 0, cudaStream_t(stream)>>>(base, n, S);
  return int(cudaGetLastError());
}

// bonds per block of the boundary kernels (one warp each)
int boundary_bonds_per_block(int cap) { (void)cap; return kBoundaryWarps; }

size_t boundary_smem(int cap) { return size_t(kZigBytes) + size_t(2 * kBoundaryWarps) * size_t(cap) * 8; }

int prepare_boundary(int cap) {
  cudaError_t e = cudaFuncSetAttribute(k_boundary, cudaFuncAttributeMaxDynamicSharedMemorySize, int(boundary_smem(cap)));
  if (e) return int(e);
  return int(cudaFuncSetAttribute(k_boundary_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(boundary_smem(cap))));
}

int launch_boundary_batch(const Dev* devs, const BatchBase* base, const int2* work, int n_work, int it, int dir,
                          int cap, void* stream) {
  if (n_work <= 0) return 0;
  k_boundary_batch<<<n_work, 32 * kBoundaryWarps, boundary_smem(cap), cudaStream_t(stream)>>>(devs, base, work, it,
                                                                                            dir, cap);
  return int(cudaGetLastError());
}

int launch_boundary(const Dev& d, int dir, void* stream) {
  const long long n = dir == 0 ? (long long)d.ndx * d.Ly : (long long)d.ndy * d.Lx;
  if ((dir == 0 && d.ndx < 2) || (dir == 1 && d.ndy < 2)) return 0;
  cudaError_t e = cudaFuncSetAttribute(k_boundary, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(boundary_smem(d.cap)));
  if (e) return int(e);
  k_boundary<<<blocks_for(n, kBoundaryWarps), 32 * kBoundaryWarps, boundary_smem(d.cap), cudaStream_t(stream)>>>(d, dir);
  return int(cudaGetLastError());
}

// Scratch of pmwa_rho_slices_static: the rho values of one call live here
// between the kernel and the copy to the host, instead of in the caller's
// arena.  Every GPU that loads the library holds this array until the
// process exits.  Calls that overlap on the GPU share it and race; each call
// overwrites all N*K values it returns, so nothing needs clearing between
// calls (the array keeps the last call's contents).
constexpr size_t kRhoStaticMax = size_t(1) << 20;  // doubles (8 MiB)
static __device__ __align__(256) double g_rho_scratch[kRhoStaticMax];

// Device address of g_rho_scratch on the current device, looked up once per
// device (in host code the symbol is only a host-side stand-in).
static double* rho_scratch_address(int* status) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static double* addr[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) { *status = PMWA_ECUDA; return nullptr; }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_rho_scratch) != cudaSuccess || !p) { *status = PMWA_ECUDA; return nullptr; }
    addr[dev] = static_cast<double*>(p);
  }
  *status = PMWA_OK;
  return addr[dev];
}

int rho_slices_static(const Dev& d, int K, double* host_out, void* stream) {
  if (K < 1 || !host_out) return PMWA_EINVAL;
  if (size_t(d.N) * size_t(K) > kRhoStaticMax) return PMWA_EINVAL;
  int st = PMWA_OK;
  double* scratch = rho_scratch_address(&st);
  if (!scratch) return st;
  k_rho<<<blocks_for(d.N, 128), 128, 0, cudaStream_t(stream)>>>(d, K, scratch);
  if (cudaGetLastError() != cudaSuccess) return PMWA_ECUDA;
  if (cudaMemcpyAsync(host_out, scratch, size_t(d.N) * size_t(K) * sizeof(double), cudaMemcpyDeviceToHost,
                      cudaStream_t(stream)) != cudaSuccess)
    return PMWA_ECUDA;
  if (cudaStreamSynchronize(cudaStream_t(stream)) != cudaSuccess) return PMWA_ECUDA;
  return PMWA_OK;
}

// Supplement S-I equal-time correlators from the worm densities rho[i*K+k]:
// blockIdx.y = r - 1 (r = 1..rmax) accumulates sum_{i,k} rho_i rho_{i+r x}
// into sums[r-1] and rho_i rho_{i+r y} into sums[rmax + r - 1]; blockIdx.y =
// rmax accumulates the plaquette product rho_i rho_{i+x} rho_{i+y}
// rho_{i+x+y} into sums[2 rmax].  Sites strided over blockIdx.x.
__global__ void k_green(int Lx, int Ly, int K, int rmax, const double* __restrict__ rho, double* sums) {
  const int N = Lx * Ly;
  const int r = int(blockIdx.y) + 1;
  double ax = 0.0, ay = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int x = i % Lx, y = i / Lx;
    const double* ri = rho + size_t(i) * K;
    if (r <= rmax) {
      const double* rx = rho + size_t((x + r) % Lx + Lx * y) * K;
      const double* ry = rho + size_t(x + Lx * ((y + r) % Ly)) * K;
      for (int k = 0; k < K; ++k) { ax = fma(ri[k], rx[k], ax); ay = fma(ri[k], ry[k], ay); }
    } else {
      const double* r1 = rho + size_t((x + 1) % Lx + Lx * y) * K;
      const double* r2 = rho + size_t(x + Lx * ((y + 1) % Ly)) * K;
      const double* r3 = rho + size_t((x + 1) % Lx + Lx * ((y + 1) % Ly)) * K;
      for (int k = 0; k < K; ++k) ax = fma(ri[k] * r1[k], r2[k] * r3[k], ax);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_down_sync(0xffffffffu, ax, o);
    ay += __shfl_down_sync(0xffffffffu, ay, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (r <= rmax) { atomicAdd(sums + (r - 1), ax); atomicAdd(sums + rmax + r - 1, ay); }
    else atomicAdd(sums + 2 * rmax, ax);
  }
}

int launch_green(int Lx, int Ly, int K, int rmax, const double* rho, double* sums, void* stream) {
  const int N = Lx * Ly;
  const int bx = N < 256 * 152 ? blocks_for(N, 256) : 152;
  k_green<<<dim3(bx, rmax + 1), 256, 0, cudaStream_t(stream)>>>(Lx, Ly, K, rmax, rho, sums);
  return int(cudaGetLastError());
}

// The generator every kernel draws from, applied to listed counters and keys
// (compared on the host with published known-answer vectors).
__global__ void k_philox(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, long long n) {
  const long long j = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t* c = in + 6 * j;
  const P4 b = philox(c[0], c[1], c[2], c[3], c[4], c[5]);
  out[4 * j] = b.x;
  out[4 * j + 1] = b.y;
  out[4 * j + 2] = b.z;
  out[4 * j + 3] = b.w;
}

int launch_philox(const uint32_t* in, uint32_t* out, int64_t n, void* stream) {
  if (n <= 0) return 0;
  k_philox<<<blocks_for(n, 128), 128, 0, cudaStream_t(stream)>>>(in, out, (long long)n);
  return int(cudaGetLastError());
}

int launch_rho(const Dev& d, int K, double* out, void* stream) {
  k_rho<<<blocks_for(d.N, 128), 128, 0, cudaStream_t(stream)>>>(d, K, out);
  return int(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Invariants of a worldline configuration with worms (Steps 3-5 keep them):
// per site, the count fits the slot; every key is a bond leg (tags 0..5) or
// a worm (7); times strictly increase; the state is continuous around the
// circle (the state above an event is the state below the next one) and the
// base state is the state above the last event; a leg's tag names a bond of
// its site; the bond's other site holds the partner leg at the same time;
// the vertex conserves particles, s0 + s1 = s2 + s3.  One warp per site,
// lanes over its events; a partner is found by bisection in at most cap
// keys, so every read stays inside the slots whatever the configuration.
// out = min over failing sites of site << 4 | code (lowest code at a site).
__device__ __forceinline__ int find_pk(const uint64_t* K, int n, uint64_t pk) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (kpk(K[mid]) < pk) lo = mid + 1; else hi = mid;
  }
  return (lo < n && kpk(K[lo]) == pk) ? lo : -1;
}

__global__ void k_check(const __grid_constant__ Dev d, unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  const long long s = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (s >= d.N) return;
  const uint32_t c = d.cntA[s];
  const int n = cnt_n(c);
  int bad = kCheckNone;
  if (n > d.cap) {
    bad = kCheckCapacity;
  } else {
    const uint64_t* K = d.keyA + size_t(s) * d.cap;
    for (int k = lane; k < n; k += 32) {
      const uint64_t key = K[k];
      const uint64_t nx = K[(k + 1 == n) ? 0 : k + 1];
      const int t = ktag(key);
      int b = kCheckNone;
      if (t == 6) b = kCheckTag;
      else if (k + 1 < n && kpk(nx) <= kpk(key)) b = kCheckOrder;
      else if (kab(key) != kbl(nx)) b = kCheckContinuity;
      else if (k + 1 == n && cnt_base(c) != kab(key)) b = kCheckBase;
      else if (t != 7) {
        int dir;
        const int a = leg_lower(d, int(s), t, &dir);
        const int o = (a == int(s)) ? site_step(d, a, dir, +1) : a;
        if (bond_tag(d, a, dir) != t) {
          b = kCheckBond;
        } else {
          const int no = min(cnt_n(d.cntA[o]), d.cap);
          const uint64_t* KO = d.keyA + size_t(o) * d.cap;
          const int ko = find_pk(KO, no, kpk(key));
          if (ko < 0) {
            b = kCheckPartner;
          } else {
            const uint64_t va = (a == int(s)) ? key : KO[ko], vb = (a == int(s)) ? KO[ko] : key;
            if (kbl(va) + kbl(vb) != kab(va) + kab(vb)) b = kCheckConservation;
          }
        }
      }
      bad = min(bad, b);
    }
  }
  for (int o = 16; o > 0; o >>= 1) bad = min(bad, __shfl_xor_sync(0xffffffffu, bad, o));
  if (lane == 0 && bad != kCheckNone)
    atomicMin(out, (static_cast<unsigned long long>(s) << 4) | static_cast<unsigned long long>(bad));
}

int launch_check(const Dev& d, unsigned long long* out, void* stream) {
  if (cudaMemsetAsync(out, 0xff, sizeof(unsigned long long), cudaStream_t(stream)) != cudaSuccess)
    return int(cudaGetLastError());
  const long long threads = static_cast<long long>(d.N) * 32;
  k_check<<<blocks_for(threads, 256), 256, 0, cudaStream_t(stream)>>>(d, out);
  return int(cudaGetLastError());
}

}  // namespace pmwa
