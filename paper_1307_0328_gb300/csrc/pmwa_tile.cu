// pmwa_tile.cu -- Steps 3-6 of one MC sweep in a single kernel: one CTA per
// domain, the domain's vertex legs and worms resident in shared memory.
//
//   phase 1  Step 3 candidates, one thread per bond of the domain, written to
//            a shared pool (the current configuration is read from HBM/L2,
//            prefetched into L2 by bulk copies at kernel start)
//   phase 2  per site: the kept vertex legs of the current configuration
//            merged in time order with the new ones into the shared leg array
//   phase 3  Step 4, one thread per site: worms of every interval (Eq. 1)
//            into the shared worm table; each worm records its site and the
//            index of the vertex leg just below it (its interval)
//   phase 4  Step 5, N_cycle passes of the shifted sub-block schedule: worms
//            grouped by sub-block, each group's worms moved in label order
//            (Eq. 2) by rounds of moves whose intervals do not meet, which
//            gives the moves made one by one; vertex legs never move in
//            Step 5, so a move is a handful of shared-memory reads and two
//            bit flips
//   phase 5  legs and worms merged per site into the next configuration in
//            HBM, with the Step-6 counters and the Supplement S-I estimator
//
// The arithmetic and the order of every random draw are those of the
// deterministic specification, so the result is bit-identical to the CPU
// reference for every domain layout.
#include <cuda_runtime.h>

#include <algorithm>

#include "pmwa_device.cuh"

namespace pmwa {

namespace {

constexpr int kMaxCandPerBond = 128;
constexpr int kMaxWormsPerInterval = 128;
constexpr uint16_t kNone = 0xFFFF;
constexpr uint32_t kCntMask = 0x7fffffffu;
constexpr uint64_t kMask62 = kTwo62 - 1;
constexpr int kSmemLimit = 232448;  // opt-in shared memory per block on sm_103a

struct WormRec {
  uint64_t key;
  uint64_t lab;   // label (Step 4); in a Step-5 pass the move's intervals, then its wait mask
  uint16_t site;  // local site index
  uint16_t leg;   // leg array index of the delimiter just below (kNone: site without legs)
  uint16_t slab;  // temporal slab (0 without temporal domains); fixed through Step 5
  uint16_t xr;    // in a Step-5 pass: rank in the sub-block, then the round of the move
};

struct Misc {
  int pool_used;
  int nworms;
  int err;
  int where;
  int wslab[64];  // worms of each temporal slab of the domain
};

__device__ __forceinline__ int cnt_n(uint32_t c) { return int(c & kCntMask); }

// bulk prefetch of `bytes` (a multiple of 16) from a 16-byte aligned global
// address into L2 (TMA engine; no registers, no completion to wait for)
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\tcp.async.bulk.prefetch.L2.global [ga], %1;\n\t}"
               :: "l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ int cnt_base(uint32_t c) { return int(c >> 31); }

__device__ __forceinline__ void tile_fail(Misc* m, int code, int where) {
  if (atomicCAS(&m->err, 0, code) == 0) m->where = where;
}

// exclusive scan of a[0..n) in place (a[n] receives the total); all threads
__device__ int block_scan(int* a, int n, int* wsum) {
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, wid = t >> 5, nw = T >> 5;
  const int chunk = (n + T - 1) / T;
  const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += a[i];
  int v = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) wsum[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < nw) ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    if (lane < nw) wsum[lane] = w;
  }
  __syncthreads();
  int run = v - sum + (wid ? wsum[wid - 1] : 0);
  for (int i = lo; i < hi; ++i) { const int x = a[i]; a[i] = run; run += x; }
  const int total = wsum[nw - 1];
  __syncthreads();
  if (t == 0) a[n] = total;
  __syncthreads();
  return total;
}

struct Tile {
  const Dev* d;
  uint64_t* th;
  int* off;        // [nds + 1] start of each site's legs in leg[]
  uint8_t* base;   // [nds] state of a site without legs
  int* bcnt;       // [2 nds] candidates per bond of the domain
  int* boff;       // [2 nds] their start in pool[]
  Misc* misc;
  uint64_t* leg;   // [legcap]
  uint8_t* wcnt;   // [legcap] worms in the interval just above each leg
  uint16_t* part;  // [legcap] index of the partner leg of each leg's vertex (kNone: none in the domain)
  uint64_t* pool;  // [poolcap] (aliases the worm table)
  WormRec* W;      // [wcap]
  uint16_t* idx;   // [wcap] worms grouped by sub-block (a pass) or by site (output)
  uint16_t* ord;   // [wcap] worm indices in label order (lab, site, key)
  uint16_t* wsb;   // [wcap] sub-block of the k-th worm in label order (a pass)
  uint16_t* wrk;   // [wcap] rank of the k-th worm inside its sub-block (a pass)
  uint64_t* rw;    // [2 wcap] Philox words of each grouped position (a pass)
  int* bkt;        // [max(nsub, nds) + 1]
  uint16_t* cnt;   // [warps x groups] per 32-worm chunk: pass stamp << 8 | worms of group u
  int* fill;       // [max(nsub, nds)]
  int16_t* nbr;    // [6 nds] per leg tag: partner site << 1 | lower-site bit, -1 off-domain
  uint8_t* tinfo;  // [6 nds] per leg tag: 1 = lower site of the bond, 2 = bond leaves the domain
  uint16_t* sub;   // [4 nds] sub-block of each site for offset pattern pass & 3
  int* soff;       // [nds + 1] start of each site's events in old[] (when staged)
  uint64_t* old;   // [oldcap] the domain's current configuration (when staged)
  int* wmo;        // [nds + 1] on-the-fly windows: start of each site's old worms in wm[]
  uint64_t* wm;    // [wcap] grid points of the current configuration's worms, by site
  bool staged;
  int x0, y0, nds, nsub;
  int ngrp;  // Step-5 chains: sub-blocks x temporal slabs

  __device__ int gsite(int li) const { return (x0 + li % d->dom_x) + d->Lx * (y0 + li / d->dom_x); }
  // current events of local site li (global site s): the staged copy or HBM
  __device__ const uint64_t* okeys(int li, int s) const {
    return staged ? old + soff[li] : d->keyA + size_t(s) * d->cap;
  }
  __device__ int lsite(int s) const { return (s % d->Lx - x0) + d->dom_x * (s / d->Lx - y0); }
  __device__ int sub_of(int li, int pass) const {
    const int B = d->sub_block;
    const int ox = (B && B < d->dom_x) ? (pass & 1) * (B / 2) : 0;
    const int oy = (B && B < d->dom_y) ? ((pass >> 1) & 1) * (B / 2) : 0;
    const int bx = sb_axis(li % d->dom_x, d->dom_x, B, d->ndx, ox);
    const int by = sb_axis(li / d->dom_x, d->dom_y, B, d->ndy, oy);
    return bx + sb_slots(d->dom_x, B, d->ndx) * by;
  }
};

// On-the-fly vertex generation (the paper's closing discussion of
// extensions): with d.win_half > 0 the vertex phase of a bond is confined to
// the grid points within win_half of a worm of the current configuration on
// either of its two sites (cyclic).  R depends on the worms alone, which
// Step 3 does not move, so the restricted heat bath keeps the distribution.
__device__ __forceinline__ bool in_win(const Tile& T, int li, uint64_t pos) {
  const uint64_t half = T.d->win_half;
  for (int k = T.wmo[li]; k < T.wmo[li + 1]; ++k) {
    const uint64_t a = (pos - T.wm[k]) & (kTwo59 - 1), b = (T.wm[k] - pos) & (kTwo59 - 1);
    if (min(a, b) <= half) return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// phase 1: Step 3 candidates of bond (a, dir) from the current configuration
// (with OTF, only inside the windows of the bond's local sites la, lb)
template <bool OTF>
__device__ int bond_candidates(const Dev& d, const ZigTab& z, int a, int dir, const uint64_t* KA, const uint64_t* KB,
                               uint64_t* buf, int cap, int* bad, const Tile* T, int la, int lb) {
  const int b = site_step(d, a, dir, +1);
  const uint64_t tag = uint64_t(bond_tag(d, a, dir));
  const uint32_t ca = d.cntA[a], cb = d.cntA[b];
  const int nA = cnt_n(ca), nB = cnt_n(cb);
  Stream s;
  s.init(d.key0, d.key1, uint32_t(2 * a + dir), c2_word(kVertex, 0, d.replica), d.sweep);
  int n = 0, ia = 0, ib = 0;
  uint64_t pos = 0;
  bool first = true;
  for (;;) {
    const uint64_t E = zig_exp(z, s, bad);
    if (*bad) break;
    const uint64_t g = grid_gap(E, d.SVs);
    const uint64_t nxt = first ? g - 1 : pos + g;
    first = false;
    if (nxt >= kTwo59) break;
    pos = nxt;
    if (OTF && !(in_win(*T, la, pos) || in_win(*T, lb, pos))) continue;
    const uint64_t pk = (pos << 3) | tag;
    while (ia < nA && kpk(KA[ia]) < pk) ++ia;
    while (ib < nB && kpk(KB[ib]) < pk) ++ib;
    if (ia < nA && kpk(KA[ia]) == pk && kab(KA[ia]) != kbl(KA[ia])) continue;  // a kink holds the point
    const int na = nA ? kab(KA[ia ? ia - 1 : nA - 1]) : cnt_base(ca);
    const int nb = nB ? kab(KB[ib ? ib - 1 : nB - 1]) : cnt_base(cb);
    const int si = na | (nb << 1);
    if (d.TV[si] < kTwo32) {
      const uint64_t w = s.word();
      if ((w >> 32) >= d.TV[si]) continue;
    }
    if (n >= cap) { *bad = PMWA_ECAPACITY; break; }
    buf[n++] = (pk << 2) | uint64_t(na) | (uint64_t(nb) << 1);
  }
  return n;
}

// old event of local site li kept by Step 3: a kink, any leg of a bond
// between domains, and (OTF) a diagonal leg outside the windows of its bond
template <bool OTF>
__device__ __forceinline__ bool kept_leg(const Tile& T, int li, uint64_t k) {
  if (kworm(k)) return false;
  if (kab(k) != kbl(k)) return true;
  if (T.tinfo[li * 6 + ktag(k)] & 2) return true;
  if (OTF) {
    const uint64_t pos = kpk(k) >> 3;
    return !(in_win(T, li, pos) || in_win(T, T.nbr[li * 6 + ktag(k)] >> 1, pos));
  }
  return false;
}

// the four bonds of local site li: (s,x) (s,y) with s the lower site, then
// (s-x,x) (s-y,y) with s the upper site; local bond id or -1 (between domains)
__device__ __forceinline__ void site_bonds(const Tile& T, int li, int lb[4]) {
  const Dev& d = *T.d;
  const int s = T.gsite(li);
  for (int j = 0; j < 4; ++j) {
    const int dir = j & 1;
    const int a = (j < 2) ? s : site_step(d, s, dir, -1);
    lb[j] = boundary_bond(d, a, dir) ? -1 : 2 * T.lsite(a) + dir;
  }
}

// ---------------------------------------------------------------------------
// phase 4: one Step-5 move of worm seg[r] (its sub-block's worms are seg[0..n),
// and only they can sit on the sub-block's sites).
__device__ int leg_index(const Tile& T, int x, uint64_t pv) {
  const int st = T.off[x], en = T.off[x + 1];
  int lo = st, hi = en;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (kpk(T.leg[mid]) < pv) lo = mid + 1; else hi = mid;
  }
  return (lo < en && kpk(T.leg[lo]) == pv) ? lo : -1;
}

constexpr uint64_t kFpTurn = ~0ull;  // descriptor of a worm that turns round whatever the others do

// The vertex that a Step-5 move of worm w (rank r in its sub-block) in pass
// pattern q reaches, as two words.  d0: the four intervals round the vertex,
// each named by the leg index of its lower delimiter -- ia_dn, ia on the
// bond's lower site a and ib_dn, ib on its upper site b (ia, ib: the vertex's
// legs); d1: the legs ia_up, ib_up above the vertex, the bond's other site
// (not w's) and r, 16 bits each.  d0 = kFpTurn: the worm turns round whatever
// the other worms do (a site without legs, a temporal boundary, a bond to
// another domain or sub-block).  Returns PMWA_EINVARIANT when the vertex has
// no partner leg on the other site.
__device__ int move_desc(const Tile& T, const WormRec& w, int q, int r, uint64_t& d0, uint64_t& d1) {
  d0 = kFpTurn;
  d1 = 0;
  const int li = w.site;
  const int st = T.off[li], en = T.off[li + 1];
  if (st == en) return PMWA_OK;
  const int L = w.leg;
  const int iv = kdir(w.key) ? ((L + 1 == en) ? st : L + 1) : L;
  const uint64_t kv = T.leg[iv];
  if (ktag(kv) == 6) return PMWA_OK;
  const int nb = T.nbr[li * 6 + ktag(kv)];
  if (nb < 0) return PMWA_OK;
  const int pl = nb >> 1;
  if (T.sub[li * 4 + q] != T.sub[pl * 4 + q]) return PMWA_OK;
  const int ip = T.d->use_part ? (T.part[iv] == kNone ? -1 : int(T.part[iv])) : leg_index(T, pl, kpk(kv));
  if (ip < 0) return PMWA_EINVARIANT;
  const bool li_a = nb & 1;  // li is the bond's lower site
  const int al = li_a ? li : pl, bl = li_a ? pl : li;
  const int ia = li_a ? iv : ip, ib = li_a ? ip : iv;
  const int sa = T.off[al], ea = T.off[al + 1], sb = T.off[bl], eb = T.off[bl + 1];
  const int ia_dn = (ia == sa) ? ea - 1 : ia - 1, ib_dn = (ib == sb) ? eb - 1 : ib - 1;
  const int ia_up = (ia + 1 == ea) ? sa : ia + 1, ib_up = (ib + 1 == eb) ? sb : ib + 1;
  d0 = uint64_t(ia_dn) | (uint64_t(ia) << 16) | (uint64_t(ib_dn) << 32) | (uint64_t(ib) << 48);
  d1 = uint64_t(ia_up) | (uint64_t(ib_up) << 16) | (uint64_t(pl) << 32) | (uint64_t(r) << 48);
  return PMWA_OK;
}

// A Step-5 move of worm w = T.W[seg[r]] (key, local site li and leg L as
// read at the start of the pass: only its own move changes them) that
// reaches the vertex of its descriptor (d0 != kFpTurn); seg[0..n) are the
// worms of its sub-block, the only ones that can sit on the sub-block's
// sites.  The worm reverses at another worm ahead of it in its interval;
// otherwise it enters the vertex v with probability L_min / L_i (word0 >> 32
// against the exact ratio), leaves by leg j (threshold table, low half of
// word0) and lands on a uniform worm grid point of leg j (mulhi of word1)
// heading away from v.  Leg l of v runs from v to the nearest event on its
// site and side (another vertex leg or worm, the moving worm excluded; the
// whole circle if none).  Legs are unique to their sites, so a worm's
// interval is named by its leg alone.  The legs and worm counts the move
// reads are loaded together up front; the vertex's two legs are updated in
// registers and stored once.
__device__ int tile_move_d(const Tile& T, WormRec& w, uint64_t key, int li, int L, uint64_t d0, uint64_t d1,
                           const uint16_t* seg, int n, int r, uint64_t w0, uint64_t w1) {
  const bool up = kdir(key);
  const int ia_dn = int(d0 & 0xffff), ia = int((d0 >> 16) & 0xffff);
  const int ib_dn = int((d0 >> 32) & 0xffff), ib = int(d0 >> 48);
  const int ia_up = int(d1 & 0xffff), ib_up = int((d1 >> 16) & 0xffff), pl = int((d1 >> 32) & 0xffff);
  const bool li_a = (L == ia || L == ia_dn);  // the worm sits on the bond's lower site
  const uint64_t kL = T.leg[L], va = T.leg[ia], vb = T.leg[ib];
  const uint64_t kad = T.leg[ia_dn], kbd = T.leg[ib_dn], kau = T.leg[ia_up], kbu = T.leg[ib_up];
  const int cL = T.wcnt[L], cia = T.wcnt[ia], cib = T.wcnt[ib], ciad = T.wcnt[ia_dn], cibd = T.wcnt[ib_dn];
  const uint64_t pL = kpk(kL);
  const uint64_t my = (kpk(key) - pL) & kMask62;
  if (cL > 1) {  // other worms share the interval: is one of them ahead?
    for (int k = 0; k < n; ++k) {
      const WormRec& o = T.W[seg[k]];
      if (k == r || int(o.leg) != L) continue;
      const uint64_t off = (kpk(o.key) - pL) & kMask62;
      if (up ? off > my : off < my) { w.key = key ^ 2u; return PMWA_OK; }
    }
  }
  const uint64_t pv = kpk(va);
  const int al = li_a ? li : pl, bl = li_a ? pl : li;
  const uint64_t pa_dn = kpk(kad), pb_dn = kpk(kbd);
  // offsets from v up to the nearest object above, and from the lower leg up
  // to the highest worm of the interval below v
  uint64_t ua = (ia_up == ia) ? kTwo62 : ((kpk(kau) - pv) & kMask62);
  uint64_t ub = (ib_up == ib) ? kTwo62 : ((kpk(kbu) - pv) & kMask62);
  uint64_t da = 0, db = 0;
  bool fa = false, fb = false;
  // worms (other than this one) in the four intervals around v?
  int others = cia + cib + (ia_dn != ia ? ciad : 0) + (ib_dn != ib ? cibd : 0) - 1;
  for (int k = 0; k < n && others > 0; ++k) {
    if (k == r) continue;
    const WormRec& o = T.W[seg[k]];
    const int lg = o.leg;
    if (lg != ia && lg != ib && lg != ia_dn && lg != ib_dn) continue;
    --others;
    const uint64_t po = kpk(o.key);
    if (lg == ia) { const uint64_t x = (po - pv) & kMask62; if (x < ua) ua = x; }
    if (lg == ib) { const uint64_t x = (po - pv) & kMask62; if (x < ub) ub = x; }
    if (lg == ia_dn) { const uint64_t x = (po - pa_dn) & kMask62; if (!fa || x > da) { da = x; fa = true; } }
    if (lg == ib_dn) { const uint64_t x = (po - pb_dn) & kMask62; if (!fb || x > db) { db = x; fb = true; } }
  }
  const uint64_t L2 = wpts(pv, (pv + ua) & kMask62);
  const uint64_t L3 = wpts(pv, (pv + ub) & kMask62);
  const uint64_t L0 = wpts(fa ? ((pa_dn + da) & kMask62) : pa_dn, pv);
  const uint64_t L1 = wpts(fb ? ((pb_dn + db) & kMask62) : pb_dn, pv);
  const int i = li_a ? (up ? 0 : 2) : (up ? 1 : 3);
  const uint64_t Li = (i == 0) ? L0 : (i == 1) ? L1 : (i == 2) ? L2 : L3;
  const uint64_t Lmin = min(min(L0, L1), min(L2, L3));
  // enter iff z1 * L_i < L_min * 2^32 (96-bit comparison)
  const uint64_t z1 = w0 >> 32, z0 = w0 & 0xffffffffull;
  const uint64_t ph = __umul64hi(z1, Li), plo = z1 * Li;
  const uint64_t qh = Lmin >> 32, ql = Lmin << 32;
  if (!(ph < qh || (ph == qh && plo < ql))) { w.key = key ^ 2u; return PMWA_OK; }
  const int S = kbl(va) | (kbl(vb) << 1) | (kab(va) << 2) | (kab(vb) << 3);
  const uint64_t* th = T.th + (S * 4 + i) * 4;
  const uint64_t t0 = th[0], t1 = th[1], t2 = th[2];
  const int j = (z0 < t0) ? 0 : (z0 < t1) ? 1 : (z0 < t2) ? 2 : 3;
  // the worm leaves leg i and takes leg j: flip their states
  uint64_t na = va, nb = vb;
  if (i & 1) nb ^= (i < 2) ? 2u : 1u; else na ^= (i < 2) ? 2u : 1u;
  if (j & 1) nb ^= (j < 2) ? 2u : 1u; else na ^= (j < 2) ? 2u : 1u;
  T.leg[ia] = na;
  T.leg[ib] = nb;
  const int ix = (j & 1) ? ib : ia;
  const uint64_t vx = (j & 1) ? nb : na;
  const uint64_t Lj = (j == 0) ? L0 : (j == 1) ? L1 : (j == 2) ? L2 : L3;
  const uint64_t o = __umul64hi(w1, Lj);
  const int nl = (j >= 2) ? ix : ((j & 1) ? ib_dn : ia_dn);
  w.key = (j >= 2) ? wkey((wm_above(pv) + o) & (kTwo59 - 1), 1, kab(vx) ^ 1)
                   : wkey((wm_below(pv) + kTwo59 - o) & (kTwo59 - 1), 0, kbl(vx));
  T.wcnt[L] -= 1;
  T.wcnt[nl] += 1;
  // site and leg in one store: a move of the same pass that runs beside this
  // one reads either the old or the new pair
  *reinterpret_cast<uint32_t*>(&w.site) = uint32_t((j & 1) ? bl : al) | (uint32_t(nl) << 16);
  return PMWA_OK;
}

// per-phase cycle counters (profiling only): thread 0 adds the cycles since
// the last tick to counter k
__device__ __forceinline__ void phase_tick(const Dev& d, int k, long long& t) {
  if (d.phase_cycles && threadIdx.x == 0) {
    const long long now = clock64();
    atomicAdd(d.phase_cycles + k, (unsigned long long)(now - t));
    t = now;
  }
}

// Step-5 chain of a worm in pass pattern q: its sub-block times N_beta plus
// its temporal slab (a worm never leaves its slab: it turns round at the
// boundaries and every leg ends there)
__device__ __forceinline__ int worm_group(const Tile& T, const WormRec& w, int q) {
  return int(T.sub[w.site * 4 + q]) * T.d->ntau + int(w.slab);
}

// ---------------------------------------------------------------------------
// Rounds of independent moves.  In a pass the worms of one sub-block move one
// after another in label order, and a move reads and writes nothing but its
// own worm and the four intervals round the vertex it reaches: their worm
// counts, the worms in them and the states of the vertex's two legs.  A worm
// that turns round whatever the others do changes nothing another move
// reads.  So a move need wait only for the earlier moves of its sub-block
// whose intervals meet its own: rounds that run every move whose such
// predecessors have run give exactly the configuration of the moves made one
// by one.
constexpr int kNear = 47;  // predecessors a wait mask names one by one
constexpr uint64_t kNearMask = (1ull << kNear) - 1;
constexpr uint16_t kPending = 0xFFFF;

// do two sets of four intervals (16-bit leg indices) share one?
__device__ __forceinline__ bool fp_meet(uint64_t a, uint64_t b) {
  const uint32_t a0 = uint32_t(a), a1 = uint32_t(a >> 32), b0 = uint32_t(b), b1 = uint32_t(b >> 32);
  const uint32_t c0 = __byte_perm(b0, 0, 0x1032), c1 = __byte_perm(b1, 0, 0x1032);  // halves swapped
  return (__vcmpeq2(a0, b0) | __vcmpeq2(a0, c0) | __vcmpeq2(a0, b1) | __vcmpeq2(a0, c1) | __vcmpeq2(a1, b0) |
          __vcmpeq2(a1, c0) | __vcmpeq2(a1, b1) | __vcmpeq2(a1, c1)) != 0;
}

// The moves of one pass (all threads).  On entry the grouped order idx[]
// (position p = fill[u] + r holds the r-th worm of group u), each position's
// move descriptor in rw[2p], rw[2p + 1], each worm's group in lab and
// kPending in xr are in place.  First each worm's wait mask goes to lab:
// bit i (i < kNear) = wait for position p - 1 - i, bits kNear.. = the group,
// bit 63 = also wait for every position of the group more than kNear before
// it.  Then rounds until every worm has moved, each move drawing Philox
// block r of stream (domain * groups + u, c2) and recording its round in
// xr.  Ends with a barrier.
__device__ void pass_rounds(const Tile& T, int dom, int nw, uint32_t c2) {
  const Dev& d = *T.d;
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int p = tid; p < nw; p += NT) {
    WormRec& w = T.W[T.idx[p]];
    const uint64_t f = T.rw[2 * p];
    uint64_t m = w.lab << kNear;
    if (f != kFpTurn) {
      const int r = int(T.rw[2 * p + 1] >> 48);
      for (int i = 0; i < r; ++i) {
        const uint64_t g = T.rw[2 * (p - 1 - i)];
        if (g != kFpTurn && fp_meet(f, g)) m |= (i < kNear) ? (1ull << i) : (1ull << 63);
      }
    }
    w.lab = m;
  }
  __syncthreads();
  for (int round = 0;; ++round) {
    int pending = 0;
    for (int p = tid; p < nw; p += NT) {
      WormRec& w = T.W[T.idx[p]];
      if (w.xr != kPending) continue;
      const uint64_t d0 = T.rw[2 * p];
      if (d0 == kFpTurn) {
        w.key ^= 2u;
        w.xr = uint16_t(round);
        continue;
      }
      const uint64_t d1 = T.rw[2 * p + 1], m = w.lab;
      const int r = int(d1 >> 48), u = int((m >> kNear) & 0xffff);
      bool ready = true;
      for (uint64_t b = m & kNearMask; b && ready; b &= b - 1)
        ready = T.W[T.idx[p - __ffsll((long long)b)]].xr < round;
      if (ready && (m >> 63))
        for (int j = p - r; j < p - kNear && ready; ++j) ready = T.W[T.idx[j]].xr < round;
      if (!ready) {
        pending = 1;
        continue;
      }
      const P4 b = philox(uint32_t(r), uint32_t(dom * T.ngrp + u), c2, d.sweep, d.key0, d.key1);
      const int rc = tile_move_d(T, w, w.key, w.site, w.leg, d0, d1, T.idx + (p - r), T.fill[u + 1] - T.fill[u], r,
                                 uint64_t(b.x) | (uint64_t(b.y) << 32), uint64_t(b.z) | (uint64_t(b.w) << 32));
      if (rc) tile_fail(T.misc, rc, 5);
      w.xr = uint16_t(round);
    }
    if (!__syncthreads_or(pending)) {
      if (d.phase_cycles && tid == 0) atomicAdd(d.phase_cycles + 7, (unsigned long long)(round + 1));
      break;
    }
    if (round >= nw) {  // (each round moves the first waiting worm of every group: never taken)
      if (tid == 0) tile_fail(T.misc, PMWA_EINVARIANT, 7);
      break;
    }
  }
}

__device__ __forceinline__ bool worm_less(const WormRec& a, const WormRec& b) {
  if (a.lab != b.lab) return a.lab < b.lab;
  if (a.site != b.site) return a.site < b.site;
  return a.key < b.key;
}

__device__ __forceinline__ void add128(uint64_t& lo, uint64_t& hi, uint64_t blo, uint64_t bhi) {
  const uint64_t s = lo + blo;
  hi += bhi + (s < lo ? 1 : 0);
  lo = s;
}

// Label order of the nw worms of the domain, (lab, site, key) ascending,
// into ord[]: a counting sort on the top bits of the (uniform 63-bit)
// labels into nbk <= max(nsub, nds) buckets, then each worm's rank inside
// its bucket.  Uses bkt/fill as bucket counters and idx as scratch.
__device__ void label_order(const Tile& T, int nw, int* wsum) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const int cap = max(T.ngrp, T.nds);
  int B = 0;
  while ((2 << B) <= cap && (1 << B) < nw) ++B;
  const int nbk = 1 << B;
  for (int i = tid; i <= nbk; i += NT) T.bkt[i] = 0;
  __syncthreads();
  for (int w = tid; w < nw; w += NT) atomicAdd(&T.bkt[B ? int(T.W[w].lab >> (63 - B)) : 0], 1);
  __syncthreads();
  block_scan(T.bkt, nbk, wsum);
  for (int i = tid; i < nbk; i += NT) T.fill[i] = T.bkt[i];
  __syncthreads();
  for (int w = tid; w < nw; w += NT)
    T.idx[atomicAdd(&T.fill[B ? int(T.W[w].lab >> (63 - B)) : 0], 1)] = uint16_t(w);
  __syncthreads();
  for (int w = tid; w < nw; w += NT) {
    const int b = B ? int(T.W[w].lab >> (63 - B)) : 0;
    const int lo = T.bkt[b], hi = T.bkt[b + 1];
    int r = 0;
    for (int j = lo; j < hi; ++j) r += worm_less(T.W[T.idx[j]], T.W[w]);
    T.ord[lo + r] = uint16_t(w);
  }
  __syncthreads();
}

// One warp (lane = threadIdx.x < 32) groups the nw worms of pass pattern q
// by sub-block, keeping label order inside each group: for the worms in
// label order, 32 at a time, the sub-block u of each (wsb), its rank among
// the worms of u met so far (wrk; equal sub-blocks in a chunk found with
// __match_any_sync, running counts in bkt[]), then fill[u] = first slot of
// sub-block u (exclusive scan of the counts) and bkt[] cleared.
__device__ void rank_pass(const Tile& T, int nw, int q, int lane) {
  const unsigned lt = (1u << lane) - 1u;
  for (int k0 = 0; k0 < nw; k0 += 32) {
    const int k = k0 + lane;
    const int u = (k < nw) ? worm_group(T, T.W[T.ord[k]], q) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, u);
    const int base = (u >= 0) ? T.bkt[u] : 0;
    __syncwarp();
    if (u >= 0) {
      T.wsb[k] = uint16_t(u);
      T.wrk[k] = uint16_t(base + __popc(peers & lt));
      if ((peers & lt) == 0) T.bkt[u] = base + __popc(peers);
    }
    __syncwarp();
  }
  const int n = T.ngrp;
  const int chunk = (n + 31) / 32;
  const int lo = min(n, lane * chunk), hi = min(n, lo + chunk);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += T.bkt[i];
  int v = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += x;
  }
  int run = v - sum;
  for (int i = lo; i < hi; ++i) {
    const int x = T.bkt[i];
    T.fill[i] = run;
    run += x;
    T.bkt[i] = 0;
  }
  if (lane == 31) T.fill[n] = v;
}

// The grouping of rank_pass by the whole block, for nw <= blockDim.x worms,
// in two halves around a block barrier (called by every thread).  Warp c ranks the
// 32 worms of chunk c of the label order among themselves (__match_any_sync)
// and its group leaders record the chunk's count of each sub-block in
// cnt[c][u], stamped with pass_stamp(pass) (an entry with another stamp
// counts 0; the table is cleared every 255 passes, so a stale stamp never
// matches).
// After the barrier every worm adds the counts of the earlier chunks to its
// rank, while one warp forms fill[] from the totals: the last warp when it
// holds no worms, else warp 0 (whose worms add nothing).  The worm of thread
// k = threadIdx.x gets its sub-block u (-1: no worm) and rank r; fill comes
// out as rank_pass makes it (after a barrier); bkt[] is scratch.
__device__ __forceinline__ int pass_stamp(int pass) { return ((pass % 255) + 1) << 8; }

// (before the barrier: the chunk ranks and counts)
__device__ void rank_chunk(const Tile& T, int nw, int q, int pass, int& u, int& r) {
  const int tid = threadIdx.x, c = tid >> 5, lane = tid & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int W = (nw + 31) >> 5, n = T.ngrp;
  const int stamp = pass_stamp(pass);
  u = -1;
  r = 0;
  if (c < W) {  // warp-uniform
    u = (tid < nw) ? worm_group(T, T.W[T.ord[tid]], q) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, u);
    r = __popc(peers & lt);
    if (u >= 0 && (peers & lt) == 0) T.cnt[c * n + u] = uint16_t(stamp | __popc(peers));
  }
}

// (after the barrier: the earlier chunks' counts, and fill[])
__device__ void rank_finish(const Tile& T, int nw, int pass, int u, int& r) {
  const int tid = threadIdx.x, c = tid >> 5, lane = tid & 31;
  const int W = (nw + 31) >> 5, n = T.ngrp;
  const int stamp = pass_stamp(pass);
  if (c > 0 && u >= 0) {
    for (int c2 = 0; c2 < c; ++c2) {
      const int v = T.cnt[c2 * n + u];
      if ((v & ~0xff) == stamp) r += v & 0xff;
    }
  }
  const int nwarps = int(blockDim.x) >> 5;
  if (c == (W < nwarps ? nwarps - 1 : 0)) {
    const int chunk = (n + 31) / 32;
    const int lo = min(n, lane * chunk), hi = min(n, lo + chunk);
    int sum = 0;
    for (int i = lo; i < hi; ++i) {
      int tot = 0;
      for (int c2 = 0; c2 < W; ++c2) {
        const int v = T.cnt[c2 * n + i];
        if ((v & ~0xff) == stamp) tot += v & 0xff;
      }
      T.bkt[i] = tot;
      sum += tot;
    }
    int v = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += x;
    }
    int run = v - sum;
    for (int i = lo; i < hi; ++i) {
      T.fill[i] = run;
      run += T.bkt[i];
      T.bkt[i] = 0;
    }
    if (lane == 31) T.fill[n] = v;
  }
}

// One pass when every worm has a thread (32 < nw <= blockDim.x; called by
// every thread, ends with a barrier).  Thread k holds the k-th worm of the
// label order from its grouping to its move: the worm's key, site and leg,
// its move descriptor, its rank r in its group u, its wait mask and its
// Philox block r of stream (domain * groups + u, c2) stay in registers.
// Other threads read only the descriptor's intervals (rw[at], for the wait
// masks) and the round of each position's move (wsb[at], kPending until it
// has moved), at its grouped position at = fill[u] + r.  The wait mask:
// bit i < 63 = wait for position at - 1 - i; bit 63 = also wait for every
// position of the group at least 64 before.  tclk: the phase clock (set-up
// to counter 5, moves to counter 6).
__device__ void pass_fast(const Tile& T, int dom, int nw, int q, int pass, uint32_t c2, long long& tclk) {
  const Dev& d = *T.d;
  const int tid = threadIdx.x, NT = blockDim.x;
  if (pass > 0 && pass % 255 == 0) {  // the stamps start over: no entry may carry one
    for (int i = tid; i < (NT >> 5) * T.ngrp; i += NT) T.cnt[i] = 0;
    __syncthreads();
  }
  int u, r;
  rank_chunk(T, nw, q, pass, u, r);
  const bool act = u >= 0;
  int wi = 0, li = 0, L = 0, rc = PMWA_OK;
  uint64_t key = 0, d0 = kFpTurn, d1 = 0;
  if (act) {
    wi = T.ord[tid];
    const WormRec& w = T.W[wi];
    key = w.key;
    li = w.site;
    L = w.leg;
    rc = move_desc(T, w, q, 0, d0, d1);
  }
  __syncthreads();
  rank_finish(T, nw, pass, u, r);
  __syncthreads();
  int at = 0, lo = 0, n = 0;
  uint64_t w0 = 0, w1 = 0;
  if (act) {
    lo = T.fill[u];
    n = T.fill[u + 1] - lo;
    at = lo + r;
    T.idx[at] = uint16_t(wi);
    T.rw[at] = d0;
    T.wsb[at] = kPending;
    if (rc) tile_fail(T.misc, rc, 5);
    if (d0 != kFpTurn) {
      const P4 b = philox(uint32_t(r), uint32_t(dom * T.ngrp + u), c2, d.sweep, d.key0, d.key1);
      w0 = uint64_t(b.x) | (uint64_t(b.y) << 32);
      w1 = uint64_t(b.z) | (uint64_t(b.w) << 32);
    }
  }
  __syncthreads();
  phase_tick(d, 5, tclk);
  uint64_t m = 0;
  if (act && d0 != kFpTurn)
    for (int i = 0; i < r; ++i) {
      const uint64_t g = T.rw[at - 1 - i];
      if (g != kFpTurn && fp_meet(d0, g)) m |= (i < 63) ? (1ull << i) : (1ull << 63);
    }
  bool done = !act;
  for (int round = 0;; ++round) {
    int pending = 0;
    if (!done) {
      bool ready = true;
      for (uint64_t b = m & ~(1ull << 63); b && ready; b &= b - 1) ready = T.wsb[at - __ffsll((long long)b)] < round;
      if (ready && (m >> 63))
        for (int j = lo; j < at - 63 && ready; ++j) ready = T.wsb[j] < round;
      if (ready) {
        WormRec& w = T.W[wi];
        if (d0 == kFpTurn) {
          w.key = key ^ 2u;
        } else {
          const int rc2 = tile_move_d(T, w, key, li, L, d0, d1, T.idx + lo, n, r, w0, w1);
          if (rc2) tile_fail(T.misc, rc2, 5);
        }
        T.wsb[at] = uint16_t(round);
        done = true;
      } else {
        pending = 1;
      }
    }
    if (!__syncthreads_or(pending)) {
      if (d.phase_cycles && tid == 0) atomicAdd(d.phase_cycles + 7, (unsigned long long)(round + 1));
      break;
    }
    if (round >= nw) {  // (each round moves the first waiting worm of every group: never taken)
      if (tid == 0) tile_fail(T.misc, PMWA_EINVARIANT, 7);
      break;
    }
  }
  phase_tick(d, 6, tclk);
}

// All N_cycle passes of a domain holding nw <= 32 worms, run by one warp
// (lane = threadIdx.x < 32) with no block barrier.  Lane k holds the k-th
// worm in label order; __match_any_sync over the groups gives each worm its
// rank r in its group, and the r-th move of a group draws Philox block r,
// as in the block-wide passes.  Each lane forms its move's descriptor (the
// intervals go through rw[lane]); a lane waits for the lanes of its group of
// lower rank whose intervals meet its own, and rounds move every lane whose
// waits are over (at most 32 rounds: the first waiting lane of each group
// waits for nobody), which gives each group's moves made one by one in rank
// order.  Returns a status (the same for all lanes).
__device__ int small_passes(const Tile& T, int dom, int nw, int lane) {
  const Dev& d = *T.d;
  const unsigned lt = (1u << lane) - 1u;
  const bool act = lane < nw;
  const int w = act ? T.ord[lane] : 0;
  for (int pass = 0; pass < d.n_cycle; ++pass) {
    const int q = pass & 3;
    const int u = act ? worm_group(T, T.W[w], q) : 0x7fffffff;
    const unsigned peers = __match_any_sync(0xffffffffu, u);
    const int r = __popc(peers & lt), n = __popc(peers);
    int less = 0;  // worms of groups numbered below u: the start of u's group
    for (int j = 0; j < 32; ++j) less += (__shfl_sync(0xffffffffu, u, j) < u) ? 1 : 0;
    int rc = PMWA_OK, li = 0, L = 0;
    uint64_t key = 0, d0 = kFpTurn, d1 = 0, w0 = 0, w1 = 0;
    if (act) {
      T.idx[less + r] = uint16_t(w);
      const WormRec& wr = T.W[w];
      key = wr.key;
      li = wr.site;
      L = wr.leg;
      rc = move_desc(T, wr, q, r, d0, d1);
      if (d0 != kFpTurn) {
        const P4 b = philox(uint32_t(r), uint32_t(dom * T.ngrp + u), c2_word(kScatter, uint32_t(pass), d.replica),
                            d.sweep, d.key0, d.key1);
        w0 = uint64_t(b.x) | (uint64_t(b.y) << 32);
        w1 = uint64_t(b.z) | (uint64_t(b.w) << 32);
      }
      T.rw[lane] = d0;
    }
    __syncwarp();
    unsigned wait = 0;  // lanes this move waits for
    if (act && d0 != kFpTurn)
      for (unsigned m = peers & lt; m; m &= m - 1) {
        const int j = __ffs(int(m)) - 1;
        const uint64_t g = T.rw[j];
        if (g != kFpTurn && fp_meet(d0, g)) wait |= 1u << j;
      }
    bool moved = !act;
    unsigned done = __ballot_sync(0xffffffffu, moved);
    while (done != 0xffffffffu) {
      if (!moved && (wait & ~done) == 0) {
        WormRec& wr = T.W[w];
        if (d0 == kFpTurn) {
          wr.key = key ^ 2u;
        } else if (rc == PMWA_OK) {
          rc = tile_move_d(T, wr, key, li, L, d0, d1, T.idx + less, n, r, w0, w1);
        }
        moved = true;
      }
      __syncwarp();
      done = __ballot_sync(0xffffffffu, moved);
    }
    const unsigned bad = __ballot_sync(0xffffffffu, rc != PMWA_OK);
    if (bad) return __shfl_sync(0xffffffffu, rc, __ffs(int(bad)) - 1);
    __syncwarp();
  }
  return PMWA_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Where the sources of a site's Step-3 merge start and end for one part of
// its circle: the old events [o0, o1), the new legs of its four bonds
// [s_j, e_j) of each run, the temporal boundaries [t0, t1).  h = -1: the
// whole circle; h = 0 / 1: the time keys below / from 2^61.
struct MergeRange {
  int o0, o1, s0, e0, s1, e1, s2, e2, s3, e3, t0, t1;
};

__device__ __forceinline__ MergeRange merge_range(const Tile& T, const uint64_t* KO, int nO, const int lb[4],
                                                  int h) {
  const Dev& d = *T.d;
  const uint64_t cut = 1ull << 61;
  const int n0 = lb[0] >= 0 ? T.bcnt[lb[0]] : 0, n1 = lb[1] >= 0 ? T.bcnt[lb[1]] : 0;
  const int n2 = lb[2] >= 0 ? T.bcnt[lb[2]] : 0, n3 = lb[3] >= 0 ? T.bcnt[lb[3]] : 0;
  const int NB = d.ntau > 1 ? d.ntau : 0;
  MergeRange R{0, nO, 0, n0, 0, n1, 0, n2, 0, n3, 0, NB};
  if (h < 0) return R;
  // (a candidate c of the pool has the time key c >> 2 = kpk(c))
  const int xo = slot_lower(KO, nO, cut);
  const int x0 = n0 ? slot_lower(T.pool + T.boff[lb[0]], n0, cut) : 0;
  const int x1 = n1 ? slot_lower(T.pool + T.boff[lb[1]], n1, cut) : 0;
  const int x2 = n2 ? slot_lower(T.pool + T.boff[lb[2]], n2, cut) : 0;
  const int x3 = n3 ? slot_lower(T.pool + T.boff[lb[3]], n3, cut) : 0;
  int xt = 0;
  while (xt < NB && tb_pk(d, xt) < cut) ++xt;
  if (h == 0) { R.o1 = xo; R.e0 = x0; R.e1 = x1; R.e2 = x2; R.e3 = x3; R.t1 = xt; }
  else { R.o0 = xo; R.s0 = x0; R.s1 = x1; R.s2 = x2; R.s3 = x3; R.t0 = xt; }
  return R;
}

// The Step-3 merge of one part of site li's circle into the leg table from
// position o: the kept old events, the new legs of its four bonds and the
// temporal boundaries (tag-6 delimiters whose state above and below is the
// worldline's state there in the current configuration; Step 3 changes no
// state), in time order.  The site is the lower site of bonds 0 and 1 (its
// state in bit 0 of a candidate) and the upper site of bonds 2 and 3 (bit 1).
template <bool OTF>
__device__ __forceinline__ void merge_site(const Tile& T, int li, const uint64_t* KO, int nO, int base0,
                                           const int lb[4], const MergeRange& R, int o) {
  const Dev& d = *T.d;
  // each run's next candidate (h) and how many remain (m)
  const uint64_t* q0 = T.pool + (lb[0] >= 0 ? T.boff[lb[0]] : 0) + R.s0;
  const uint64_t* q1 = T.pool + (lb[1] >= 0 ? T.boff[lb[1]] : 0) + R.s1;
  const uint64_t* q2 = T.pool + (lb[2] >= 0 ? T.boff[lb[2]] : 0) + R.s2;
  const uint64_t* q3 = T.pool + (lb[3] >= 0 ? T.boff[lb[3]] : 0) + R.s3;
  int m0 = R.e0 - R.s0, m1 = R.e1 - R.s1, m2 = R.e2 - R.s2, m3 = R.e3 - R.s3;
  uint64_t h0 = m0 ? q0[0] : 0, h1 = m1 ? q1[0] : 0, h2 = m2 ? q2[0] : 0, h3 = m3 ? q3[0] : 0;
  int io = R.o0, ib = R.t0;
  uint64_t tb = ib < R.t1 ? tb_pk(d, ib) : 0;
  for (;;) {
    uint64_t ko = 0;
    while (io < R.o1 && !kept_leg<OTF>(T, li, ko = KO[io])) ++io;
    uint64_t best = ~0ull;
    int src = -1;
    if (io < R.o1) { best = kpk(ko); src = 4; }
    if (m0 && (h0 >> 2) < best) { best = h0 >> 2; src = 0; }
    if (m1 && (h1 >> 2) < best) { best = h1 >> 2; src = 1; }
    if (m2 && (h2 >> 2) < best) { best = h2 >> 2; src = 2; }
    if (m3 && (h3 >> 2) < best) { best = h3 >> 2; src = 3; }
    if (ib < R.t1 && tb < best) { best = tb; src = 5; }
    if (src < 0) break;
    uint64_t key;
    switch (src) {
      case 4: key = ko; ++io; break;
      case 5: {
        const uint64_t bst = uint64_t(slot_state(KO, nO, base0, best));
        key = (best << 2) | (bst << 1) | bst;
        if (++ib < R.t1) tb = tb_pk(d, ib);
        break;
      }
      case 0: { const uint64_t st = h0 & 1; key = ((h0 >> 2) << 2) | (st << 1) | st; if (--m0) h0 = *++q0; break; }
      case 1: { const uint64_t st = h1 & 1; key = ((h1 >> 2) << 2) | (st << 1) | st; if (--m1) h1 = *++q1; break; }
      case 2: { const uint64_t st = (h2 >> 1) & 1; key = ((h2 >> 2) << 2) | (st << 1) | st; if (--m2) h2 = *++q2; break; }
      default: { const uint64_t st = (h3 >> 1) & 1; key = ((h3 >> 2) << 2) | (st << 1) | st; if (--m3) h3 = *++q3; break; }
    }
    T.leg[o++] = key;
  }
}

template <bool OTF>
__device__ __forceinline__ void tile_body(const Dev& d, const int dom, const int stop, unsigned char* sm,
                                          int* wsum) {
  Tile T;
  T.d = &d;
  T.th = reinterpret_cast<uint64_t*>(sm + d.sm_th);
  T.off = reinterpret_cast<int*>(sm + d.sm_off);
  T.base = reinterpret_cast<uint8_t*>(sm + d.sm_base);
  T.bcnt = reinterpret_cast<int*>(sm + d.sm_bcnt);
  T.boff = reinterpret_cast<int*>(sm + d.sm_boff);
  T.misc = reinterpret_cast<Misc*>(sm + d.sm_misc);
  T.leg = reinterpret_cast<uint64_t*>(sm + d.sm_leg);
  T.wcnt = reinterpret_cast<uint8_t*>(sm + d.sm_wcnt);
  T.part = reinterpret_cast<uint16_t*>(sm + d.sm_part);
  T.pool = reinterpret_cast<uint64_t*>(sm + d.sm_pool);
  T.W = reinterpret_cast<WormRec*>(sm + d.sm_worm);
  T.idx = reinterpret_cast<uint16_t*>(sm + d.sm_idx);
  T.ord = reinterpret_cast<uint16_t*>(sm + d.sm_ord);
  T.wsb = reinterpret_cast<uint16_t*>(sm + d.sm_wsb);
  T.wrk = reinterpret_cast<uint16_t*>(sm + d.sm_wrk);
  T.rw = reinterpret_cast<uint64_t*>(sm + d.sm_rw);
  T.bkt = reinterpret_cast<int*>(sm + d.sm_bkt);
  T.cnt = reinterpret_cast<uint16_t*>(sm + d.sm_cnt);
  T.fill = reinterpret_cast<int*>(sm + d.sm_fill);
  T.nbr = reinterpret_cast<int16_t*>(sm + d.sm_nbr);
  T.tinfo = reinterpret_cast<uint8_t*>(sm + d.sm_tinfo);
  T.sub = reinterpret_cast<uint16_t*>(sm + d.sm_sub);
  T.soff = reinterpret_cast<int*>(sm + d.sm_soff);
  T.old = reinterpret_cast<uint64_t*>(sm + d.sm_old);
  T.staged = false;
  T.x0 = (dom % d.ndx) * d.dom_x;
  T.y0 = (dom / d.ndx) * d.dom_y;
  T.nds = d.dom_x * d.dom_y;
  T.nsub = sb_slots(d.dom_x, d.sub_block, d.ndx) * sb_slots(d.dom_y, d.sub_block, d.ndy);
  T.ngrp = T.nsub * d.ntau;
  const int tid = threadIdx.x, NT = blockDim.x, nds = T.nds;
  Misc* misc = T.misc;

  long long tclk = clock64();
  // the domain's current event lists on their way into L2 before the scans
  // of Step 3 reach them: one bulk prefetch per site of its used slots (a
  // list starts 64-byte aligned; its length rounded up to 16 bytes stays
  // within the site's cap, a multiple of 8 keys)
  for (int li = tid; li < nds; li += NT) {
    const int s = T.gsite(li), n = cnt_n(d.cntA[s]);
    if (n) prefetch_l2(d.keyA + size_t(s) * d.cap, uint32_t((n * 8 + 15) & ~15));
  }
  const ZigTab Z = zig_stage(sm + d.sm_zig, d.zig_cap, d.worm_tries);
  for (int k = tid; k < 256; k += NT) T.th[k] = d.TH[k];
  if (tid == 0) { misc->pool_used = 0; misc->nworms = 0; misc->err = 0; misc->where = 0; }
  for (int k = tid; k < d.ntau; k += NT) misc->wslab[k] = 0;
  // per-site tables: bond partners by leg tag, sub-blocks by offset pattern
  for (int li = tid; li < nds; li += NT) {
    for (int t = 0; t < 6; ++t) { T.nbr[li * 6 + t] = -1; T.tinfo[li * 6 + t] = 0; }
    const int s = T.gsite(li);
    for (int j = 0; j < 4; ++j) {
      const int dir = j & 1;
      const int a = (j < 2) ? s : site_step(d, s, dir, -1);
      const int tg = bond_tag(d, a, dir);
      const bool out = boundary_bond(d, a, dir);
      T.tinfo[li * 6 + tg] = uint8_t((j < 2 ? 1 : 0) | (out ? 2 : 0));
      if (out) continue;
      const int other = (j < 2) ? site_step(d, s, dir, +1) : a;
      T.nbr[li * 6 + tg] = int16_t((T.lsite(other) << 1) | (j < 2 ? 1 : 0));
    }
    for (int q = 0; q < 4; ++q) T.sub[li * 4 + q] = uint16_t(T.sub_of(li, q));
  }
  __syncthreads();

  // stage the domain's current configuration in shared memory (one warp per
  // site, coalesced), so that the scans of phases 1-2 do not wait on HBM/L2
  if (d.oldcap > 0) {
    for (int li = tid; li < nds; li += NT) T.soff[li] = cnt_n(d.cntA[T.gsite(li)]);
    __syncthreads();
    if (block_scan(T.soff, nds, wsum) <= d.oldcap) {
      const int lane = tid & 31;
      for (int li = tid >> 5; li < nds; li += NT >> 5) {
        const uint64_t* KO = d.keyA + size_t(T.gsite(li)) * d.cap;
        const int st = T.soff[li], n = T.soff[li + 1] - st;
        for (int k = lane; k < n; k += 32) T.old[st + k] = KO[k];
      }
      T.staged = true;
    }
    __syncthreads();
  }

  if (OTF) {
    // the worms of the current configuration, by site: the windows of the
    // on-the-fly vertex phase
    T.wmo = reinterpret_cast<int*>(sm + d.sm_wmo);
    T.wm = reinterpret_cast<uint64_t*>(sm + d.sm_wm);
    for (int li = tid; li < nds; li += NT) {
      const int s = T.gsite(li), n = cnt_n(d.cntA[s]);
      const uint64_t* KO = T.okeys(li, s);
      int c = 0;
      for (int k = 0; k < n; ++k) c += kworm(KO[k]) ? 1 : 0;
      T.wmo[li] = c;
    }
    __syncthreads();
    if (block_scan(T.wmo, nds, wsum) > d.wcap) { if (tid == 0) tile_fail(misc, PMWA_ECAPACITY, 35); }
    __syncthreads();
    if (misc->err) goto fail;
    for (int li = tid; li < nds; li += NT) {
      const int s = T.gsite(li), n = cnt_n(d.cntA[s]);
      const uint64_t* KO = T.okeys(li, s);
      int o = T.wmo[li];
      for (int k = 0; k < n; ++k) if (kworm(KO[k])) T.wm[o++] = kpk(KO[k]) >> 3;
    }
    __syncthreads();
  }

  // ---- phase 1: Step 3 candidates per bond
  for (int lb = tid; lb < 2 * nds; lb += NT) {
    const int li = lb >> 1, dir = lb & 1;
    const int a = T.gsite(li);
    uint64_t buf[kMaxCandPerBond];
    int n = 0, bad = 0;
    if (d.has_vertices && !boundary_bond(d, a, dir)) {
      const int b = site_step(d, a, dir, +1);
      n = bond_candidates<OTF>(d, Z, a, dir, T.okeys(li, a), T.okeys(T.lsite(b), b), buf,
                               min(d.capb, kMaxCandPerBond), &bad, &T, li, T.lsite(b));
    }
    if (bad) { tile_fail(misc, bad, 31); n = 0; }
    int o = 0;
    if (n) {
      o = atomicAdd(&misc->pool_used, n);
      if (o + n > d.poolcap) { tile_fail(misc, PMWA_ECAPACITY, 32); n = 0; }
      else for (int k = 0; k < n; ++k) T.pool[o + k] = buf[k];
    }
    T.bcnt[lb] = n;
    T.boff[lb] = o;
  }
  __syncthreads();
  phase_tick(d, 0, tclk);
  if (misc->err) goto fail;

  // ---- phase 2: kept legs + new legs per site, merged in time order.  With
  // two threads a site to spare (the 512-thread CTA of a 16x16 domain) each
  // site's circle is cut at time key 2^61 and its two halves are counted and
  // merged by two threads; each half is in time order and the halves follow
  // one another, so the leg table is the one a single thread writes.  The
  // half counts go through the (not yet used) worm-count bytes as scratch.
  {
    const bool two = NT >= 2 * nds && d.legcap >= 8 * nds;
    const int units = two ? 2 * nds : nds;
    int* hc = reinterpret_cast<int*>(T.wcnt);
    for (int un = tid; un < units; un += NT) {
      const int li = two ? un % nds : un, h = two ? un / nds : -1;
      const int s = T.gsite(li);
      const uint64_t* KO = T.okeys(li, s);
      const int nO = cnt_n(d.cntA[s]);
      int lb[4];
      site_bonds(T, li, lb);
      const MergeRange R = merge_range(T, KO, nO, lb, h);
      int c = 0;
      for (int k = R.o0; k < R.o1; ++k) c += kept_leg<OTF>(T, li, KO[k]);
      c += (R.e0 - R.s0) + (R.e1 - R.s1) + (R.e2 - R.s2) + (R.e3 - R.s3) + (R.t1 - R.t0);
      if (two) hc[h * nds + li] = c;
      else T.off[li] = c;
    }
    if (two) {
      __syncthreads();
      for (int li = tid; li < nds; li += NT) T.off[li] = hc[li] + hc[nds + li];
    }
    __syncthreads();
    if (block_scan(T.off, nds, wsum) > d.legcap) { if (tid == 0) tile_fail(misc, PMWA_ECAPACITY, 33); }
    __syncthreads();
    if (misc->err) goto fail;
    for (int un = tid; un < units; un += NT) {
      const int li = two ? un % nds : un, h = two ? un / nds : -1;
      const int s = T.gsite(li);
      const uint64_t* KO = T.okeys(li, s);
      const int nO = cnt_n(d.cntA[s]);
      int lb[4];
      site_bonds(T, li, lb);
      const MergeRange R = merge_range(T, KO, nO, lb, h);
      merge_site<OTF>(T, li, KO, nO, cnt_base(d.cntA[s]), lb, R, T.off[li] + (h == 1 ? hc[li] : 0));
    }
  }
  __syncthreads();
  if (stop >= 5 && d.use_part) {
    // the partner leg of every vertex leg whose bond lies in the domain: the
    // leg with the same time on the bond's other site (legs keep their
    // places through Step 5; only their states change)
    // (legs split evenly over the threads; each vertex once, from its lower site)
    const int total = T.off[nds];
    for (int j = tid; j < total; j += NT) T.part[j] = kNone;
    __syncthreads();
    const int chunk = (total + NT - 1) / NT;
    int j = tid * chunk;
    const int jend = min(total, j + chunk);
    if (j < jend) {
      int a = 0, b = nds;  // the site of leg j: off[a] <= j < off[a + 1]
      while (a + 1 < b) {
        const int m = (a + b) >> 1;
        if (T.off[m] <= j) a = m; else b = m;
      }
      int li = a;
      for (; j < jend; ++j) {
        while (T.off[li + 1] <= j) ++li;
        const uint64_t key = T.leg[j];
        if (ktag(key) == 6) continue;  // a temporal boundary
        const int nb = T.nbr[li * 6 + ktag(key)];
        if (nb < 0 || (nb & 1) == 0) continue;
        const int ip = leg_index(T, nb >> 1, kpk(key));
        if (ip < 0) { tile_fail(misc, PMWA_EINVARIANT, 34); continue; }
        T.part[j] = uint16_t(ip);
        T.part[ip] = uint16_t(j);
      }
    }
    __syncthreads();
  }
  phase_tick(d, 1, tclk);

  if (stop >= 4) {
    // ---- phase 3: Step 4, worms of every interval (the pool is dead now)
    for (int li = tid; li < nds; li += NT) {
      const int s = T.gsite(li);
      const int st = T.off[li], nl = T.off[li + 1] - st;
      Stream rs;
      rs.init(d.key0, d.key1, uint32_t(s), c2_word(kRegen, 0, d.replica), d.sweep);
      uint64_t offs[kMaxWormsPerInterval];
      int bad = 0;
      if (nl == 0) {
        const int s0 = int(rs.word() >> 63);
        T.base[li] = uint8_t(s0);
        const int n = sample_worms<kMaxWormsPerInterval>(Z, rs, kTwo59, 0, d.SWs, d.SWI, offs, &bad);
        if (!bad && n > 0) {
          const int o = atomicAdd(&misc->nworms, n);
          atomicAdd(&misc->wslab[0], n);
          if (o + n > d.wcap) bad = PMWA_ECAPACITY;
          for (int k = 0; k < n && !bad; ++k) {
            const uint64_t w = rs.word();
            T.W[o + k] = WormRec{wkey(offs[k], int(w & 1), s0 ^ 1 ^ (k & 1)), w >> 1, uint16_t(li), kNone, 0, 0};
          }
        }
      } else {
        // (the state of a site whose delimiters are temporal boundaries only
        // and which keeps no worm: all its boundary states are equal)
        T.base[li] = uint8_t(kab(T.leg[st]));
        for (int k = 0; k < nl && !bad; ++k) {
          const uint64_t lo = T.leg[st + k], hi = T.leg[st + (k + 1 == nl ? 0 : k + 1)];
          const uint64_t M = wpts(kpk(lo), kpk(hi));
          const int p = kab(lo), sigma = p ^ kbl(hi);
          const int n = sample_worms<kMaxWormsPerInterval>(Z, rs, M, sigma, d.SWs, d.SWI, offs, &bad);
          T.wcnt[st + k] = uint8_t(n > 0 ? min(n, 255) : 0);
          if (n > 255) bad = PMWA_ECAPACITY;
          if (bad || n <= 0) continue;
          const int o = atomicAdd(&misc->nworms, n);
          if (o + n > d.wcap) { bad = PMWA_ECAPACITY; break; }
          const uint64_t m0 = wm_above(kpk(lo));
          // an interval lies inside one temporal slab (boundaries delimit it)
          const int sl = slab_of_m(d, m0);
          atomicAdd(&misc->wslab[sl], n);
          for (int j = 0; j < n; ++j) {
            const uint64_t w = rs.word();
            T.W[o + j] = WormRec{wkey((m0 + offs[j]) & (kTwo59 - 1), int(w & 1), p ^ 1 ^ (j & 1)), w >> 1,
                                 uint16_t(li), uint16_t(st + k), uint16_t(sl), 0};
          }
        }
      }
      if (bad) tile_fail(misc, bad, 4);
    }
    __syncthreads();
    phase_tick(d, 2, tclk);
    if (misc->err) goto fail;

    // ---- phase 4: Step 5
    if (stop >= 5) {
      const int nw = misc->nworms;
      if (nw > 0) label_order(T, nw, wsum);
      // The shifted sub-block schedule: in pass p every worm moves once,
      // inside the sub-block of offset pattern p & 3 that holds its site, in
      // label order; the r-th move of sub-block u draws Philox block r of
      // stream (unit = domain * n_sub + u, scatter | pass).
      for (int u = tid; u < T.ngrp; u += NT) T.bkt[u] = 0;
      for (int i = tid; i < (NT >> 5) * T.ngrp; i += NT) T.cnt[i] = 0;  // no stamp of this sweep
      __syncthreads();
      if (nw > 0 && nw <= 32) {  // few worms: one warp, no block barrier per pass
        if (tid < 32) {
          const int rc = small_passes(T, dom, nw, tid);
          if (rc && tid == 0) tile_fail(misc, rc, 5);
        }
        __syncthreads();
        if (misc->err) goto fail;
      }
      for (int pass = 0; pass < (nw > 32 ? d.n_cycle : 0); ++pass) {  // no worms: nothing moves
        const int q = pass & 3;
        const uint32_t c2 = c2_word(kScatter, uint32_t(pass), d.replica);
        if (nw <= NT) {  // all warps, one chunk each, one worm a thread
          pass_fast(T, dom, nw, q, pass, c2, tclk);
          if (misc->err) goto fail;
          continue;
        }
        {
          if (tid < 32) rank_pass(T, nw, q, tid);
          __syncthreads();
          for (int k = tid; k < nw; k += NT) {
            const int u = T.wsb[k], r = T.wrk[k], at = T.fill[u] + r;
            T.idx[at] = T.ord[k];
            WormRec& w = T.W[T.ord[k]];
            const int rc = move_desc(T, w, q, r, T.rw[2 * at], T.rw[2 * at + 1]);
            if (rc) tile_fail(misc, rc, 5);
            w.lab = uint64_t(u);
            w.xr = kPending;
          }
        }
        __syncthreads();
        phase_tick(d, 5, tclk);
        if (misc->err) goto fail;
        pass_rounds(T, dom, nw, c2);
        phase_tick(d, 6, tclk);
        if (misc->err) goto fail;
      }
      phase_tick(d, 3, tclk);
    }
  }

  // ---- phase 5: next configuration + Step 6
  {
    const int nw = (stop >= 4) ? misc->nworms : 0;
    if (stop >= 4) {
      for (int li = tid; li <= nds; li += NT) T.bkt[li] = 0;
      __syncthreads();
      for (int w = tid; w < nw; w += NT) atomicAdd(&T.bkt[T.W[w].site], 1);
      __syncthreads();
      block_scan(T.bkt, nds, wsum);
      for (int li = tid; li < nds; li += NT) T.fill[li] = T.bkt[li];
      __syncthreads();
      for (int w = tid; w < nw; w += NT) T.idx[atomicAdd(&T.fill[T.W[w].site], 1)] = uint16_t(w);
      __syncthreads();
    }
    uint64_t nv = 0, nk = 0, nwc = 0, olo = 0, ohi = 0, qlo = 0, qhi = 0;
    double q = 0.0;
    for (int li = tid; li < nds; li += NT) {
      const int s = T.gsite(li);
      const int st = T.off[li], nl = T.off[li + 1] - st;
      uint64_t* OUT = d.keyB + size_t(s) * d.cap;
      const uint64_t* KO = d.keyA + size_t(s) * d.cap;
      const int nO = cnt_n(d.cntA[s]);
      uint16_t* seg = nullptr;
      int nws = 0;
      if (stop >= 4) {
        seg = T.idx + T.bkt[li];
        nws = T.bkt[li + 1] - T.bkt[li];
        for (int p = 1; p < nws; ++p) {  // worms of the site in time order
          const uint16_t v = seg[p];
          int r = p - 1;
          while (r >= 0 && T.W[v].key < T.W[seg[r]].key) { seg[r + 1] = seg[r]; --r; }
          seg[r + 1] = v;
        }
      }
      // merge legs with worms (stop 3: the old worms); the occupied time of
      // the intervals between consecutive events is summed as they are
      // written (Step 6), the interval round the circle after the last one
      int il = 0, iw = 0, io = 0, no = 0, nww = 0;
      bool bad = false;
      uint64_t occ = 0, first_pk = 0, prev = 0;
      for (;;) {
        uint64_t wk = ~0ull;
        if (stop >= 4) { if (iw < nws) wk = T.W[seg[iw]].key; }
        else {
          while (io < nO && !kworm(KO[io])) ++io;
          if (io < nO) wk = KO[io];
        }
        const uint64_t lk = il < nl ? T.leg[st + il] : ~0ull;
        if (lk == ~0ull && wk == ~0ull) break;
        uint64_t key;
        if (kpk(lk) < kpk(wk) || wk == ~0ull) {
          key = lk;
          ++il;
          if (ktag(key) == 6) continue;  // a temporal boundary is no event
        } else {
          key = wk;
          ++nww;
          if (stop >= 4) ++iw; else ++io;
        }
        if (no >= d.cap) { bad = true; break; }
        if (no == 0) first_pk = kpk(key);
        else if (kab(prev)) occ += (kpk(key) - kpk(prev)) & kMask62;
        prev = key;
        OUT[no++] = key;
      }
      if (bad) { tile_fail(misc, PMWA_ECAPACITY, 6); continue; }
      int base;
      if (no) base = kab(OUT[no - 1]);
      else base = (stop >= 4) ? T.base[li] : cnt_base(d.cntA[s]);
      d.cntB[s] = uint32_t(no) | (uint32_t(base) << 31);
      if (stop < 6) continue;
      // Step 6, per site: occupied time (at most 2^62 a site, summed in 128
      // bits), worms; a site without legs is one interval of sigma = 0
      if (no == 0) occ = base ? kTwo62 : 0;
      else if (no == 1) occ = kab(prev) ? kTwo62 : 0;
      else if (kab(prev)) occ += (first_pk - kpk(prev)) & kMask62;
      add128(olo, ohi, occ, 0);
      nwc += uint64_t(nww);
      if (nl == 0) {
        uint64_t v;
        if (xg_fix(0, kTwo59, d.XQ, v)) add128(qlo, qhi, v, 0);
        else q += xg_sigma(0, double(kTwo59) * d.XW);
      }
    }
    if (stop >= 6) {
      // Step 6, per interval (legs split evenly over the threads): vertex
      // and kink counts, and the improved <Q> sum of x g_sigma(x), in fixed
      // point (exact sum) where x < 1/2, else in binary64
      const int total = T.off[nds];
      const int chunk = (total + NT - 1) / NT;
      int j = tid * chunk;
      const int jend = min(total, j + chunk);
      if (j < jend) {
        int a = 0, b = nds;  // the site of leg j: off[a] <= j < off[a + 1]
        while (a + 1 < b) {
          const int m = (a + b) >> 1;
          if (T.off[m] <= j) a = m; else b = m;
        }
        int li = a;
        for (; j < jend; ++j) {
          while (T.off[li + 1] <= j) ++li;
          const uint64_t lo = T.leg[j];
          const uint64_t hi = T.leg[(j + 1 == T.off[li + 1]) ? T.off[li] : j + 1];
          if (ktag(lo) < 6 && (T.tinfo[li * 6 + ktag(lo)] & 1)) { ++nv; if (kab(lo) != kbl(lo)) ++nk; }
          const uint64_t I = wpts(kpk(lo), kpk(hi));
          const int sg = kab(lo) ^ kbl(hi);
          uint64_t v;
          if (xg_fix(sg, I, d.XQ, v)) add128(qlo, qhi, v, 0);
          else q += xg_sigma(sg, __ull2double_rn(I) * d.XW);
        }
      }
      q += __ull2double_rn(qhi) * 4.0 + __ull2double_rn(qlo) * 0x1p-62;
    }
    if (stop >= 6) {
      for (int o = 16; o > 0; o >>= 1) {
        nv += __shfl_down_sync(0xffffffffu, nv, o);
        nk += __shfl_down_sync(0xffffffffu, nk, o);
        nwc += __shfl_down_sync(0xffffffffu, nwc, o);
        const uint64_t blo = __shfl_down_sync(0xffffffffu, olo, o);
        const uint64_t bhi = __shfl_down_sync(0xffffffffu, ohi, o);
        add128(olo, ohi, blo, bhi);
        q += __shfl_down_sync(0xffffffffu, q, o);
      }
      if ((tid & 31) == 0) {
        pmwa_row* r = d.rows + d.row;
        if (nv) atomicAdd(reinterpret_cast<unsigned long long*>(&r->n_v), (unsigned long long)nv);
        if (nk) atomicAdd(reinterpret_cast<unsigned long long*>(&r->n_k), (unsigned long long)nk);
        if (nwc) atomicAdd(reinterpret_cast<unsigned long long*>(&r->n_w), (unsigned long long)nwc);
        if (olo | ohi) {
          const unsigned long long old =
              atomicAdd(reinterpret_cast<unsigned long long*>(&r->occ_lo), (unsigned long long)olo);
          const uint64_t carry = (old + olo < old) ? 1 : 0;
          if (ohi + carry)
            atomicAdd(reinterpret_cast<unsigned long long*>(&r->occ_hi), (unsigned long long)(ohi + carry));
        }
        atomicAdd(&r->q_impr, q);
      }
      if (dom == 0 && tid == 0) d.rows[d.row].sweep = d.sweep;
      if (tid == 0) {
        // worms per (space-time) domain: the fewest (kept as a complement, so
        // that the zeroed row and an atomic maximum give the minimum) and the
        // empty ones
        pmwa_row* r = d.rows + d.row;
        unsigned wmin = ~0u, empty = 0;
        for (int k = 0; k < d.ntau; ++k) {
          wmin = min(wmin, unsigned(misc->wslab[k]));
          empty += misc->wslab[k] == 0 ? 1u : 0u;
        }
        atomicMax(&r->w_dom_min, ~wmin);
        if (empty) atomicAdd(&r->dom_empty, empty);
      }
    }
    __syncthreads();
    phase_tick(d, 4, tclk);
    if (misc->err) goto fail;
  }
  return;
fail:
  if (tid == 0) set_err(d.err, misc->err, misc->where);
}

// CTAs of NT threads may use up to 128 registers a thread (512 / NT CTAs per
// SM by registers)
template <int NT, bool OTF>
__global__ void __launch_bounds__(NT, 512 / NT) k_tile(const __grid_constant__ Dev d, int stop) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int wsum[32];
  if (instance_failed(d.err)) return;
  tile_body<OTF>(d, int(blockIdx.x), stop, sm, wsum);
}

// Batched form: one CTA per (instance, domain) work item; the instance's
// parameters are copied into shared memory and advanced to sweep iteration
// `it` of the current batch call (buffers, sweep index, row).
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_tile_batch(const Dev* __restrict__ devs,
                                                   const BatchBase* __restrict__ base,
                                                   const int2* __restrict__ work, int it, int stop) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int wsum[32];
  __shared__ Dev sd;
  const int2 w = work[blockIdx.x];
  if (!base[w.x].active) return;
  if (threadIdx.x == 0) sd = at_iteration(devs[w.x], base[w.x], it);
  __syncthreads();
  if (instance_failed(sd.err)) return;
  tile_body<false>(sd, w.y, stop, sm, wsum);
}

// ---------------------------------------------------------------------------
// Shared-memory plan of one domain.  Fixed tables, then the leg table
// (legcap legs and a worm count each), then a union that holds the Step-3
// candidate pool and, beside it, the staged current configuration (phases
// 1-2), later the worm table and the Step-5 arrays.  The configuration is
// staged only when that costs no CTA per SM (CTAs per SM: the 228 KB of
// shared memory of an SM over the per-CTA size plus its 1 KB reserve).
bool plan_tile_smem(Dev* d, double legs_want, double cands_per_bond) {
  const int nds = d->dom_x * d->dom_y;
  // Step-5 chains: sub-blocks x temporal slabs
  const int nsub = sb_slots_host(d->dom_x, d->sub_block, d->ndx) * sb_slots_host(d->dom_y, d->sub_block, d->ndy) *
                   std::max(1, d->ntau);
  const int nb = std::max(nsub, nds) + 1;
  auto up16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  size_t o = 0;
  d->sm_th = int(o); o = up16(o + 256 * sizeof(uint64_t));
  d->sm_zig = int(o); o = up16(o + size_t(kZigBytes));
  d->sm_off = int(o); o = up16(o + size_t(nds + 1) * sizeof(int));
  d->sm_base = int(o); o = up16(o + size_t(nds));
  d->sm_bcnt = int(o); o = up16(o + size_t(2 * nds) * sizeof(int));
  d->sm_boff = int(o); o = up16(o + size_t(2 * nds) * sizeof(int));
  d->sm_misc = int(o); o = up16(o + sizeof(Misc));
  d->sm_nbr = int(o); o = up16(o + size_t(6 * nds) * sizeof(int16_t));
  d->sm_sub = int(o); o = up16(o + size_t(4 * nds) * sizeof(uint16_t));
  d->sm_tinfo = int(o); o = up16(o + size_t(6 * nds));
  const size_t fixed = o;
  // worm side of the union: table, index, label order, sub-block ids and
  // ranks, Philox words, two bucket arrays
  // (and the per-chunk sub-block counts of the block-wide grouping: one row
  // per warp of the domain's CTA, 16 for CTAs of 256 or 512 threads)
  const int warps = nds <= 32 ? 2 : (nds <= 96 ? 4 : 16);
  const size_t cnt_bytes = up16(size_t(warps) * size_t(nsub) * sizeof(uint16_t));
  const size_t worm_bytes = up16(size_t(d->wcap) * sizeof(WormRec)) + 4 * up16(size_t(d->wcap) * 2) +
                            up16(size_t(d->wcap) * 16) + 2 * up16(size_t(nb) * sizeof(int)) + cnt_bytes;
  // (on-the-fly windows: the worms of the current configuration by site, beside the pool)
  const size_t otf_bytes = d->win_half ? up16(size_t(nds + 1) * sizeof(int)) + up16(size_t(d->wcap) * 8) : 0;
  const size_t pool_bytes = up16(size_t(d->poolcap) * sizeof(uint64_t)) + otf_bytes;
  const long long want = std::min<long long>((long long)legs_want, 65000);
  const long long limit = (long long)kSmemLimit - 1024;
  // CTAs per SM: shared memory (1 KB the hardware reserves a CTA and up to
  // 1 KB of static shared memory), registers (up to 128 a thread: 2, 4 or 8
  // CTAs of 256, 128 or 64 threads) and the 32-CTA limit
  const long long by_regs = nds <= 32 ? 8 : (nds <= 96 ? 4 : 2);
  auto per_sm = [&](long long bytes) { return std::min(std::min((228LL * 1024) / (bytes + 2048), by_regs), 32LL); };
  // without staging
  const long long uni0 = (long long)std::max(worm_bytes, pool_bytes);
  const long long room = limit - (long long)fixed - uni0;
  if (room < 8 * 64) return false;
  // legs, their worm counts and (optionally) their partner indices
  auto legs_bytes = [&](long long c, bool part) {
    return (long long)up16(size_t(c) * 8) + (long long)up16(size_t(c)) + (part ? (long long)up16(size_t(c) * 2) : 0);
  };
  const long long capn = std::min<long long>(want, room / 9 - 16);
  const long long totn = (long long)fixed + legs_bytes(capn, false) + uni0;
  const long long capp = std::min<long long>(want, room / 11 - 16);
  const long long totp = (long long)fixed + legs_bytes(capp, true) + uni0;
  // the partner table only when it shrinks neither the leg table nor occupancy
  const bool part = capp == capn && per_sm(totp) >= per_sm(totn);
  const long long cap0 = part ? capp : capn;
  const long long tot0 = part ? totp : totn;
  // with staging: room for as many events as legs
  const long long stage = (long long)up16(size_t(nds + 1) * sizeof(int)) + (long long)up16(size_t(want) * 8);
  const long long uni1 = std::max((long long)worm_bytes, (long long)pool_bytes + stage);
  const long long tot1 = (long long)fixed + legs_bytes(want, part) + uni1;
  const bool staged = cap0 == want && tot1 <= limit && per_sm(tot1) >= per_sm(tot0);
  d->legcap = int(cap0);
  d->oldcap = staged ? int(want) : 0;
  d->sm_leg = int(o); o = up16(o + size_t(d->legcap) * sizeof(uint64_t));
  d->sm_wcnt = int(o); o = up16(o + size_t(d->legcap));
  d->use_part = part ? 1 : 0;
  d->sm_part = int(o); if (part) o = up16(o + size_t(d->legcap) * 2);
  d->sm_pool = int(o);
  d->sm_wmo = int(o + up16(size_t(d->poolcap) * sizeof(uint64_t)));
  d->sm_wm = int(d->sm_wmo + up16(size_t(nds + 1) * sizeof(int)));
  d->sm_soff = int(o + pool_bytes);
  d->sm_old = int(o + pool_bytes + up16(size_t(nds + 1) * sizeof(int)));
  d->sm_worm = int(o);
  size_t w = o + up16(size_t(d->wcap) * sizeof(WormRec));
  d->sm_idx = int(w); w = up16(w + size_t(d->wcap) * 2);
  d->sm_ord = int(w); w = up16(w + size_t(d->wcap) * 2);
  d->sm_wsb = int(w); w = up16(w + size_t(d->wcap) * 2);
  d->sm_wrk = int(w); w = up16(w + size_t(d->wcap) * 2);
  d->sm_rw = int(w); w = up16(w + size_t(d->wcap) * 16);
  d->sm_bkt = int(w); w = up16(w + size_t(nb) * sizeof(int));
  d->sm_cnt = int(w); w += cnt_bytes;
  d->sm_fill = int(w); w = up16(w + size_t(nb) * sizeof(int));
  o = std::max(w, o + pool_bytes + (staged ? size_t(stage) : 0));
  d->sm_total = int(o);
  (void)cands_per_bond;
  return d->sm_total <= kSmemLimit - 1024;
}

int upload_zig_tile(const Zig& z) { return upload_constants(z); }

// CTA sizes of the sweep kernel: small domains take small CTAs, so that many
// of them share an SM (class 0: 64 threads, 1: 128, 2: 256); a large domain
// whose plan leaves room for one CTA per SM takes 512 threads (class 3),
// which the registers then allow
int tile_class(int domain_sites, int smem) {
  if (domain_sites <= 32) return 0;
  if (domain_sites <= 96) return 1;
  return (228LL * 1024) / (static_cast<long long>(smem) + 2048) <= 1 ? 3 : 2;
}

int prepare_tile_batch(int cls, int smem) {
  cudaError_t e;
  switch (cls) {
    case 0: e = cudaFuncSetAttribute(k_tile_batch<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    case 1: e = cudaFuncSetAttribute(k_tile_batch<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    case 2: e = cudaFuncSetAttribute(k_tile_batch<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    default: e = cudaFuncSetAttribute(k_tile_batch<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
  }
  return int(e);
}

int launch_tile_batch(int cls, const Dev* devs, const BatchBase* base, const int2* work, int n_work, int smem,
                      int it, int stop, void* stream) {
  if (n_work <= 0) return 0;
  const cudaStream_t st = cudaStream_t(stream);
  switch (cls) {
    case 0: k_tile_batch<64><<<n_work, 64, smem, st>>>(devs, base, work, it, stop); break;
    case 1: k_tile_batch<128><<<n_work, 128, smem, st>>>(devs, base, work, it, stop); break;
    case 2: k_tile_batch<256><<<n_work, 256, smem, st>>>(devs, base, work, it, stop); break;
    default: k_tile_batch<512><<<n_work, 512, smem, st>>>(devs, base, work, it, stop); break;
  }
  return int(cudaGetLastError());
}

template <int NT, bool OTF>
static int launch_tile_k(const Dev& d, int stop, cudaStream_t st) {
  const cudaError_t e = cudaFuncSetAttribute(k_tile<NT, OTF>, cudaFuncAttributeMaxDynamicSharedMemorySize, d.sm_total);
  if (e) return int(e);
  k_tile<NT, OTF><<<d.ndom, NT, d.sm_total, st>>>(d, stop);
  return int(cudaGetLastError());
}

int launch_tile(const Dev& d, int stop, void* stream) {
  const int cls = tile_class(d.dom_x * d.dom_y, d.sm_total);
  const cudaStream_t st = cudaStream_t(stream);
  const bool otf = d.win_half > 0;
  switch (cls) {
    case 0: return otf ? launch_tile_k<64, true>(d, stop, st) : launch_tile_k<64, false>(d, stop, st);
    case 1: return otf ? launch_tile_k<128, true>(d, stop, st) : launch_tile_k<128, false>(d, stop, st);
    case 2: return otf ? launch_tile_k<256, true>(d, stop, st) : launch_tile_k<256, false>(d, stop, st);
    default: return otf ? launch_tile_k<512, true>(d, stop, st) : launch_tile_k<512, false>(d, stop, st);
  }
}

}  // namespace pmwa
