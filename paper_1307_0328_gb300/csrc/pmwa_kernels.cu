// pmwa_kernels.cu -- sm_103a kernels of one PMWA Monte Carlo step.
//
//   k_boundary   Step 2 (Eq. 4) + Step 3 on the bonds between domains;
//                one thread per boundary bond, x bonds then y bonds.
//   k_step3      Step 3 (vertex phase) candidates of every other bond;
//                one thread per bond.
//   k_step34     per site: merge the kept vertex legs with the new ones and
//                draw the worms of every interval (Step 4, Eq. 1).
//   k_step5      Step 5 (Eq. 2), all N_cycle passes; one CTA per domain,
//                one thread per sub-block of the shifted sub-block schedule.
//   k_measure    Step 6: exact counters and the Supplement S-I estimator.
//
// Configuration layout in HBM: site i owns the slot key[i*cap .. i*cap+cap)
// of 64-bit event keys sorted in time, and cnt[i] = count | base << 31.
#include <cuda_runtime.h>

#include "pmwa_device.cuh"

namespace pmwa {

constexpr int kMaxWormsPerInterval = 128;
constexpr uint32_t kCntMask = 0x7fffffffu;

__device__ __forceinline__ int cnt_n(uint32_t c) { return int(c & kCntMask); }
__device__ __forceinline__ int cnt_base(uint32_t c) { return int(c >> 31); }
__device__ __forceinline__ uint32_t cnt_make(int n, int base) { return uint32_t(n) | (uint32_t(base) << 31); }

// ---------------------------------------------------------------------------
// Step 3 (vertex phase), candidates of one bond.  The bond's diagonal
// vertices are dropped (by k_step34) and new ones laid as a Bernoulli process
// of mean spacing SV = 2^59/(beta D) on its 2^59 time points, each kept with
// probability d(s)/D (u32 threshold), s the occupations of its two sites at
// that time in the current configuration; a point held by one of the bond's
// kinks is skipped.  Output: (pk << 2) | na | nb << 1, in time order.
__global__ void k_step3(Dev d) {
  const int bid = blockIdx.x * blockDim.x + threadIdx.x;
  if (bid >= 2 * d.N) return;
  const int a = bid >> 1, dir = bid & 1;
  if (boundary_bond(d, a, dir)) return;
  if (!d.has_vertices) { d.ccnt[bid] = 0; return; }
  const int b = site_step(d, a, dir, +1);
  const uint64_t tag = uint64_t(bond_tag(d, a, dir));
  const uint64_t* KA = d.keyA + size_t(a) * d.cap;
  const uint64_t* KB = d.keyA + size_t(b) * d.cap;
  const uint32_t ca = d.cntA[a], cb = d.cntA[b];
  const int nA = cnt_n(ca), nB = cnt_n(cb);
  Stream s;
  s.init(d.key0, d.key1, uint32_t(bid), c2_word(kVertex, 0, d.replica), d.sweep);
  uint64_t* out = d.cand + size_t(bid) * d.capb;
  int n = 0, bad = 0;
  int ia = 0, ib = 0;  // first event with pk >= candidate pk on a / b
  uint64_t pos = 0;
  bool first = true;
  for (;;) {
    const double E = zig_exp(s, &bad);
    if (bad) break;
    const uint64_t g = grid_gap(E, d.SV);
    const uint64_t nxt = first ? g - 1 : pos + g;
    first = false;
    if (nxt >= kTwo59) break;
    pos = nxt;
    const uint64_t pk = (pos << 3) | tag;
    while (ia < nA && kpk(KA[ia]) < pk) ++ia;
    while (ib < nB && kpk(KB[ib]) < pk) ++ib;
    if (ia < nA && kpk(KA[ia]) == pk && kab(KA[ia]) != kbl(KA[ia])) continue;  // kink holds it
    const int na = nA ? kab(KA[ia ? ia - 1 : nA - 1]) : cnt_base(ca);
    const int nb = nB ? kab(KB[ib ? ib - 1 : nB - 1]) : cnt_base(cb);
    const int si = na | (nb << 1);
    if (d.TV[si] < kTwo32) {
      const uint64_t w = s.word();
      if ((w >> 32) >= d.TV[si]) continue;
    }
    if (n >= d.capb) { bad = PMWA_ECAPACITY; break; }
    out[n++] = (pk << 2) | uint64_t(na) | (uint64_t(nb) << 1);
  }
  if (bad) set_err(d.err, bad, 3);
  d.ccnt[bid] = uint32_t(n);
}

// in-place reversal of [lo, hi) of two parallel arrays
__device__ __forceinline__ void rev2(uint64_t* k, uint64_t* l, int lo, int hi) {
  for (--hi; lo < hi; ++lo, --hi) {
    const uint64_t t = k[lo]; k[lo] = k[hi]; k[hi] = t;
    const uint64_t u = l[lo]; l[lo] = l[hi]; l[hi] = u;
  }
}

// ---------------------------------------------------------------------------
// Step 3 merge + Step 4 on one site.  The new slot is the time-ordered merge
// of the kept events of the current slot (kinks, every leg of a boundary
// bond; worms too when regen == 0) with the new diagonal vertices of the
// site's up to four non-boundary bonds.  With regen, the worms are then drawn
// interval by interval (Eq. 1): intervals between consecutive vertex legs,
// the last one wrapping round the circle; types alternate from the state
// just above the lower leg; one word per worm gives label (>> 1) and
// direction (& 1).  A site without legs is one closed interval of length
// beta with a uniformly drawn state and an even number of worms.
__global__ void k_step34(Dev d, int regen) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.N) return;
  const uint64_t* KO = d.keyA + size_t(s) * d.cap;
  const uint32_t co = d.cntA[s];
  const int nO = cnt_n(co);
  // the four bonds of s: (s,x), (s,y) with s the lower site; (s-x,x), (s-y,y)
  const uint64_t* cl[4];
  int cn[4], ci[4], cbit[4];
  for (int j = 0; j < 4; ++j) {
    const int dir = j & 1;
    const int a = (j < 2) ? s : site_step(d, s, dir, -1);
    cn[j] = 0; ci[j] = 0; cbit[j] = (j < 2) ? 0 : 1; cl[j] = nullptr;
    if (!boundary_bond(d, a, dir) && d.has_vertices) {
      const int bid = 2 * a + dir;
      cl[j] = d.cand + size_t(bid) * d.capb;
      cn[j] = int(d.ccnt[bid]);
    }
  }
  uint64_t* T = regen ? d.tmp + size_t(s) * d.cap : d.keyB + size_t(s) * d.cap;
  int nl = 0, io = 0, bad = 0;
  for (;;) {
    // next kept event of the old slot
    while (io < nO) {
      const uint64_t k = KO[io];
      if (kworm(k)) { if (!regen) break; ++io; continue; }
      if (kab(k) != kbl(k)) break;  // kink
      int dir;
      const int a = leg_lower(d, s, ktag(k), &dir);
      if (boundary_bond(d, a, dir)) break;
      ++io;  // diagonal vertex of a bond of this domain: replaced
    }
    uint64_t best = ~0ull;
    int src = -1;
    if (io < nO) { best = kpk(KO[io]); src = 4; }
    for (int j = 0; j < 4; ++j)
      if (ci[j] < cn[j]) {
        const uint64_t p = cl[j][ci[j]] >> 2;
        if (p < best) { best = p; src = j; }
      }
    if (src < 0) break;
    uint64_t key;
    if (src == 4) { key = KO[io++]; }
    else {
      const uint64_t c = cl[src][ci[src]++];
      const uint64_t st = (c >> cbit[src]) & 1;
      key = ((c >> 2) << 2) | (st << 1) | st;
    }
    if (nl >= d.cap) { bad = PMWA_ECAPACITY; break; }
    T[nl++] = key;
  }
  if (bad) { set_err(d.err, bad, 34); d.cntB[s] = cnt_make(0, cnt_base(co)); return; }
  if (!regen) {
    uint64_t* LB = d.lab + size_t(s) * d.cap;
    for (int k = 0; k < nl; ++k) LB[k] = 0;
    d.cntB[s] = cnt_make(nl, nl ? kab(T[nl - 1]) : cnt_base(co));
    return;
  }
  // Step 4
  Stream st;
  st.init(d.key0, d.key1, uint32_t(s), c2_word(kRegen, 0, d.replica), d.sweep);
  uint64_t* OUT = d.keyB + size_t(s) * d.cap;
  uint64_t* LB = d.lab + size_t(s) * d.cap;
  uint64_t offs[kMaxWormsPerInterval];
  int no = 0, base;
  if (nl == 0) {
    const int s0 = int(st.word() >> 63);
    const int n = sample_worms<kMaxWormsPerInterval>(st, kTwo59, 0, d.SW, d.SWI, offs, &bad);
    for (int k = 0; k < n && !bad; ++k) {
      const uint64_t w = st.word();
      if (no >= d.cap) { bad = PMWA_ECAPACITY; break; }
      OUT[no] = wkey(offs[k], int(w & 1), s0 ^ 1 ^ (k & 1));
      LB[no] = w >> 1;
      ++no;
    }
    base = s0;
  } else {
    int wrapped = 0;
    for (int k = 0; k < nl && !bad; ++k) {
      const uint64_t lo = T[k], hi = T[(k + 1) % nl];
      if (no >= d.cap) { bad = PMWA_ECAPACITY; break; }
      OUT[no] = lo; LB[no] = 0; ++no;
      const uint64_t M = wpts(kpk(lo), kpk(hi));
      const int p = kab(lo), sigma = p ^ kbl(hi);
      const int n = sample_worms<kMaxWormsPerInterval>(st, M, sigma, d.SW, d.SWI, offs, &bad);
      if (bad) break;
      const uint64_t m0 = wm_above(kpk(lo));
      for (int j = 0; j < n; ++j) {
        const uint64_t w = st.word();
        if (no >= d.cap) { bad = PMWA_ECAPACITY; break; }
        const uint64_t m = (m0 + offs[j]) & (kTwo59 - 1);
        if (k == nl - 1 && m < m0) ++wrapped;
        OUT[no] = wkey(m, int(w & 1), p ^ 1 ^ (j & 1));
        LB[no] = w >> 1;
        ++no;
      }
    }
    if (!bad && wrapped) {  // worms past the end of the circle belong in front
      rev2(OUT, LB, 0, no);
      rev2(OUT, LB, 0, wrapped);
      rev2(OUT, LB, wrapped, no);
    }
    base = no ? kab(OUT[no - 1]) : 0;
  }
  if (bad) { set_err(d.err, bad, 4); no = 0; }
  d.cntB[s] = cnt_make(no, base);
}

// ---------------------------------------------------------------------------
// Step 5 (worm scattering, Eq. 2).
struct WormRef {
  uint32_t site;
  uint32_t pad;
  uint64_t pk;
  uint64_t lab;
};
__device__ __forceinline__ bool wref_less(const WormRef& a, const WormRef& b) {
  if (a.lab != b.lab) return a.lab < b.lab;
  if (a.site != b.site) return a.site < b.site;
  return a.pk < b.pk;
}

// length of a vertex leg in worm grid points: from the vertex at pk pv on
// site x up (or down) to the next event other than the moving worm; the whole
// circle when there is none.
__device__ uint64_t leg_len(const Dev& d, int x, uint64_t pv, bool up, int ws, uint64_t wpk) {
  const uint64_t* K = d.keyB + size_t(x) * d.cap;
  const int n = cnt_n(d.cntB[x]);
  const int iv = slot_find(K, n, pv);
  if (iv < 0) return ~0ull;  // partner leg missing: corrupt configuration
  int j = iv;
  for (int k = 0; k < n; ++k) {
    j = up ? (j + 1 == n ? 0 : j + 1) : (j == 0 ? n - 1 : j - 1);
    if (j == iv) break;
    const uint64_t pj = kpk(K[j]);
    if (x == ws && pj == wpk) continue;
    return up ? wpts(pv, pj) : wpts(pj, pv);
  }
  return kTwo59;
}

__device__ __forceinline__ void slot_erase(uint64_t* K, uint64_t* L, int n, int at) {
  for (int k = at; k + 1 < n; ++k) { K[k] = K[k + 1]; L[k] = L[k + 1]; }
}
__device__ __forceinline__ void slot_insert(uint64_t* K, uint64_t* L, int n, int at, uint64_t key, uint64_t lab) {
  for (int k = n; k > at; --k) { K[k] = K[k - 1]; L[k] = L[k - 1]; }
  K[at] = key; L[at] = lab;
}
__device__ __forceinline__ void fix_base(const Dev& d, int x) {
  const uint32_t c = d.cntB[x];
  const int n = cnt_n(c);
  if (n) d.cntB[x] = cnt_make(n, kab(d.keyB[size_t(x) * d.cap + n - 1]));
}

// One move of the worm (ws, wpk) with the two words of its Philox block:
// reverse at a worm or at a vertex of an inactive bond; otherwise enter with
// probability L_min / L_i (word0 >> 32 against the exact ratio), leave by
// leg j from the threshold table (low half of word0), land uniformly on leg j
// (mulhi of word1) heading away from the vertex.  Returns a status.
__device__ int scatter_move(const Dev& d, const uint64_t* TH, int pass, int ws, uint64_t wpk,
                            uint64_t w0, uint64_t w1) {
  uint64_t* K = d.keyB + size_t(ws) * d.cap;
  uint64_t* L = d.lab + size_t(ws) * d.cap;
  const int n = cnt_n(d.cntB[ws]);
  const int iw = slot_find(K, n, wpk);
  if (iw < 0 || n < 2) return PMWA_EINVARIANT;
  const uint64_t key = K[iw], lab = L[iw];
  const bool up = kdir(key);
  const int ie = up ? (iw + 1 == n ? 0 : iw + 1) : (iw == 0 ? n - 1 : iw - 1);
  const uint64_t ke = K[ie];
  if (kworm(ke)) { K[iw] = key ^ 2u; return PMWA_OK; }
  int dir;
  const int a = leg_lower(d, ws, ktag(ke), &dir);
  const int b = site_step(d, a, dir, +1);
  if (boundary_bond(d, a, dir) || sb_local(d, a, pass) != sb_local(d, b, pass)) {
    K[iw] = key ^ 2u;
    return PMWA_OK;
  }
  const uint64_t pv = kpk(ke);
  const int i = (ws == a) ? (up ? 0 : 2) : (up ? 1 : 3);
  uint64_t Lg[4], Lmin = 0;
  for (int l = 0; l < 4; ++l) {
    Lg[l] = leg_len(d, (l & 1) ? b : a, pv, l >= 2, ws, wpk);
    if (Lg[l] == ~0ull) return PMWA_EINVARIANT;
    if (l == 0 || Lg[l] < Lmin) Lmin = Lg[l];
  }
  // enter iff z1 * L_i < L_min * 2^32 (96-bit comparison)
  const uint64_t z1 = w0 >> 32, z0 = w0 & 0xffffffffull;
  const uint64_t ph = __umul64hi(z1, Lg[i]), pl = z1 * Lg[i];
  const uint64_t qh = Lmin >> 32, ql = Lmin << 32;
  if (!(ph < qh || (ph == qh && pl < ql))) { K[iw] = key ^ 2u; return PMWA_OK; }
  uint64_t* KA = d.keyB + size_t(a) * d.cap;
  uint64_t* KB = d.keyB + size_t(b) * d.cap;
  const int ka = slot_find(KA, cnt_n(d.cntB[a]), pv), kb = slot_find(KB, cnt_n(d.cntB[b]), pv);
  if (ka < 0 || kb < 0) return PMWA_EINVARIANT;
  const uint64_t va = KA[ka], vb = KB[kb];
  const int S = kbl(va) | (kbl(vb) << 1) | (kab(va) << 2) | (kab(vb) << 3);
  const uint64_t* th = TH + (S * 4 + i) * 4;
  int j = 0;
  while (j < 3 && !(z0 < th[j])) ++j;
  // remove the worm, then flip the entry and exit root states of the vertex
  slot_erase(K, L, n, iw);
  d.cntB[ws] = cnt_make(n - 1, cnt_base(d.cntB[ws]));
  {
    uint64_t* Ki = (i & 1) ? KB : KA;
    const int xi = (i & 1) ? b : a;
    const int fi = slot_find(Ki, cnt_n(d.cntB[xi]), pv);
    uint64_t* Kj = (j & 1) ? KB : KA;
    const int xj = (j & 1) ? b : a;
    const int fj = slot_find(Kj, cnt_n(d.cntB[xj]), pv);
    if (fi < 0 || fj < 0) return PMWA_EINVARIANT;
    Ki[fi] ^= (i < 2) ? 2u : 1u;
    Kj[fj] ^= (j < 2) ? 2u : 1u;
  }
  const int x = (j & 1) ? b : a;
  uint64_t* KX = d.keyB + size_t(x) * d.cap;
  uint64_t* LX = d.lab + size_t(x) * d.cap;
  const int nx = cnt_n(d.cntB[x]);
  if (nx >= d.cap) return PMWA_ECAPACITY;
  const int kx = slot_find(KX, nx, pv);
  if (kx < 0) return PMWA_EINVARIANT;
  const uint64_t vx = KX[kx];
  const uint64_t o = __umul64hi(w1, Lg[j]);
  uint64_t nk;
  if (j >= 2) nk = wkey((wm_above(pv) + o) & (kTwo59 - 1), 1, kab(vx) ^ 1);
  else        nk = wkey((wm_below(pv) + kTwo59 - o) & (kTwo59 - 1), 0, kbl(vx));
  const int at = slot_lower(KX, nx, kpk(nk));
  slot_insert(KX, LX, nx, at, nk, lab);
  d.cntB[x] = cnt_make(nx + 1, cnt_base(d.cntB[x]));
  fix_base(d, a);
  fix_base(d, b);
  return PMWA_OK;
}

// One CTA per domain runs all N_cycle passes.  Per pass the domain's worms
// are bucketed by sub-block in shared memory; each thread then owns whole
// sub-blocks (their sites are touched by no other thread) and moves their
// worms in ascending label order, the r-th move using Philox block r of the
// stream (unit = domain * n_sub + sub-block, c2 = scatter | pass).
__global__ void k_step5(Dev d) {
  extern __shared__ unsigned char smem[];
  const int nsx = sb_slots(d.dom_x, d.sub_block, d.ndx), nsy = sb_slots(d.dom_y, d.sub_block, d.ndy);
  const int nsub = nsx * nsy;
  uint64_t* sTH = reinterpret_cast<uint64_t*>(smem);
  int* cnt = reinterpret_cast<int*>(sTH + 256);
  int* fill = cnt + (nsub + 1);
  WormRef* W = reinterpret_cast<WormRef*>(
      reinterpret_cast<uintptr_t>(fill + nsub + 1 + 3) & ~uintptr_t(15));
  __shared__ int s_bad;
  const int dom = blockIdx.x;
  const int x0 = (dom % d.ndx) * d.dom_x, y0 = (dom / d.ndx) * d.dom_y;
  const int nds = d.dom_x * d.dom_y;
  for (int k = threadIdx.x; k < 256; k += blockDim.x) sTH[k] = d.TH[k];
  if (threadIdx.x == 0) s_bad = 0;
  for (int pass = 0; pass < d.n_cycle; ++pass) {
    for (int k = threadIdx.x; k <= nsub; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    for (int li = threadIdx.x; li < nds; li += blockDim.x) {
      const int s = (x0 + li % d.dom_x) + d.Lx * (y0 + li / d.dom_x);
      const uint64_t* K = d.keyB + size_t(s) * d.cap;
      const int n = cnt_n(d.cntB[s]);
      int nw = 0;
      for (int k = 0; k < n; ++k) nw += kworm(K[k]);
      if (nw) atomicAdd(&cnt[sb_local(d, s, pass) + 1], nw);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int u = 0; u < nsub; ++u) cnt[u + 1] += cnt[u];
      if (cnt[nsub] > d.wcap) s_bad = PMWA_ECAPACITY;
    }
    __syncthreads();
    if (s_bad) break;
    for (int u = threadIdx.x; u < nsub; u += blockDim.x) fill[u] = cnt[u];
    __syncthreads();
    for (int li = threadIdx.x; li < nds; li += blockDim.x) {
      const int s = (x0 + li % d.dom_x) + d.Lx * (y0 + li / d.dom_x);
      const uint64_t* K = d.keyB + size_t(s) * d.cap;
      const uint64_t* L = d.lab + size_t(s) * d.cap;
      const int n = cnt_n(d.cntB[s]);
      const int u = sb_local(d, s, pass);
      for (int k = 0; k < n; ++k)
        if (kworm(K[k])) {
          const int at = atomicAdd(&fill[u], 1);
          W[at] = WormRef{uint32_t(s), 0u, kpk(K[k]), L[k]};
        }
    }
    __syncthreads();
    for (int u = threadIdx.x; u < nsub; u += blockDim.x) {
      const int lo = cnt[u], hi = cnt[u + 1];
      for (int p = lo + 1; p < hi; ++p) {  // insertion sort by (label, site, pk)
        const WormRef v = W[p];
        int q = p - 1;
        while (q >= lo && wref_less(v, W[q])) { W[q + 1] = W[q]; --q; }
        W[q + 1] = v;
      }
      Stream st;
      st.init(d.key0, d.key1, uint32_t(dom * nsub + u), c2_word(kScatter, uint32_t(pass), d.replica), d.sweep);
      for (int r = 0; r < hi - lo; ++r) {
        st.pos = 2 * uint64_t(r);
        const uint64_t w0 = st.word(), w1 = st.word();
        const int rc = scatter_move(d, sTH, pass, int(W[lo + r].site), W[lo + r].pk, w0, w1);
        if (rc) { atomicCAS(&s_bad, 0, rc); break; }
      }
    }
    __syncthreads();
    if (s_bad) break;
  }
  if (threadIdx.x == 0 && s_bad) set_err(d.err, s_bad, 5);
}

// ---------------------------------------------------------------------------
// Step 6 (measurement) on the configuration after Step 5.  Exact counters
// (vertices and kinks counted on their bond's lower site, worms, occupied
// time in units beta/2^62 as a 128-bit sum) and the Supplement S-I improved
// estimator sum_intervals x g_sigma(x), intervals between vertex legs.
__device__ __forceinline__ void add128(uint64_t& lo, uint64_t& hi, uint64_t blo, uint64_t bhi) {
  const uint64_t s = lo + blo;
  hi += bhi + (s < lo ? 1 : 0);
  lo = s;
}

__global__ void k_measure(Dev d) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t nv = 0, nk = 0, nw = 0, olo = 0, ohi = 0;
  double q = 0.0;
  if (s < d.N) {
    const uint64_t* K = d.keyB + size_t(s) * d.cap;
    const uint32_t c = d.cntB[s];
    const int n = cnt_n(c);
    if (n == 0) {
      if (cnt_base(c)) olo = kTwo62;
      const double x = __dmul_rn(double(kTwo59), d.XW);
      q = __dmul_rn(x, g_sigma(0, x));
    } else {
      int first = -1, prev = -1;
      for (int k = 0; k < n; ++k) {
        const uint64_t key = K[k];
        const uint64_t nx = kpk(K[k + 1 == n ? 0 : k + 1]);
        const uint64_t len = (n == 1) ? kTwo62 : ((nx - kpk(key)) & (kTwo62 - 1));
        if (kab(key)) olo += len;
        if (kworm(key)) { ++nw; continue; }
        int dir;
        if (leg_lower(d, s, ktag(key), &dir) == s) { ++nv; if (kab(key) != kbl(key)) ++nk; }
        if (first < 0) first = k;
        if (prev >= 0) {
          const double x = __dmul_rn(__ull2double_rn(wpts(kpk(K[prev]), kpk(key))), d.XW);
          q = __dadd_rn(q, __dmul_rn(x, g_sigma(kab(K[prev]) ^ kbl(key), x)));
        }
        prev = k;
      }
      if (first < 0) {
        const double x = __dmul_rn(double(kTwo59), d.XW);
        q = __dmul_rn(x, g_sigma(0, x));
      } else {
        const double x = __dmul_rn(__ull2double_rn(wpts(kpk(K[prev]), kpk(K[first]))), d.XW);
        q = __dadd_rn(q, __dmul_rn(x, g_sigma(kab(K[prev]) ^ kbl(K[first]), x)));
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    nv += __shfl_down_sync(0xffffffffu, nv, off);
    nk += __shfl_down_sync(0xffffffffu, nk, off);
    nw += __shfl_down_sync(0xffffffffu, nw, off);
    const uint64_t blo = __shfl_down_sync(0xffffffffu, olo, off);
    const uint64_t bhi = __shfl_down_sync(0xffffffffu, ohi, off);
    add128(olo, ohi, blo, bhi);
    q += __shfl_down_sync(0xffffffffu, q, off);
  }
  if ((threadIdx.x & 31) == 0) {
    pmwa_row* r = d.rows + d.row;
    if (nv) atomicAdd(reinterpret_cast<unsigned long long*>(&r->n_v), (unsigned long long)nv);
    if (nk) atomicAdd(reinterpret_cast<unsigned long long*>(&r->n_k), (unsigned long long)nk);
    if (nw) atomicAdd(reinterpret_cast<unsigned long long*>(&r->n_w), (unsigned long long)nw);
    if (olo | ohi) {
      const unsigned long long old =
          atomicAdd(reinterpret_cast<unsigned long long*>(&r->occ_lo), (unsigned long long)olo);
      const uint64_t carry = (old + olo < old) ? 1 : 0;
      if (ohi + carry) atomicAdd(reinterpret_cast<unsigned long long*>(&r->occ_hi), (unsigned long long)(ohi + carry));
    }
    atomicAdd(&r->q_impr, q);
  }
  if (s == 0) d.rows[d.row].sweep = d.sweep;
}

// Supplement S-I worm density at K equal-time slices tau_k = k beta / K:
// eta g_sigma(x) of the interval between vertex legs holding tau_k.
__global__ void k_rho(Dev d, int K, double* out) {
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
};

// the two legs of the vertex at pv on a site: to the next vertex leg below
// and above, worms ignored; one interval round the circle if v is alone.
__device__ bool site_legs(const uint64_t* K, int n, uint64_t pv, Legs* L) {
  const int iv = slot_find(K, n, pv);
  if (iv < 0) return false;
  int jn = iv, jp = iv;
  for (int k = 0; k < n; ++k) { jn = (jn + 1 == n) ? 0 : jn + 1; if (jn == iv || !kworm(K[jn])) break; }
  for (int k = 0; k < n; ++k) { jp = (jp == 0) ? n - 1 : jp - 1; if (jp == iv || !kworm(K[jp])) break; }
  L->single = (jn == iv);
  if (L->single) { L->plo = L->phi = pv; L->Idn = L->Iup = kTwo59; L->far_dn = L->far_up = 0; return true; }
  L->phi = kpk(K[jn]); L->far_up = kbl(K[jn]); L->Iup = wpts(pv, L->phi);
  L->plo = kpk(K[jp]); L->far_dn = kab(K[jp]); L->Idn = wpts(L->plo, pv);
  return true;
}

__device__ __forceinline__ void aslot_erase(uint64_t* K, int n, int at) {
  for (int k = at; k + 1 < n; ++k) K[k] = K[k + 1];
}
__device__ __forceinline__ void aslot_insert(uint64_t* K, int n, int at, uint64_t key) {
  for (int k = n; k > at; --k) K[k] = K[k - 1];
  K[at] = key;
}

// erase the worms strictly inside (lo, hi) going up (lo == hi: all of them)
// and draw new ones with end states p (above lo) and q (below hi).
__device__ int regen_interval(const Dev& d, Stream& st, int x, uint64_t lo, uint64_t hi, int p, int q) {
  uint64_t* K = d.keyA + size_t(x) * d.cap;
  int n = cnt_n(d.cntA[x]);
  const uint64_t span = (hi > lo) ? hi - lo : hi + kTwo62 - lo;
  for (int k = n - 1; k >= 0; --k) {
    if (!kworm(K[k])) continue;
    const uint64_t off = (kpk(K[k]) + kTwo62 - lo) & (kTwo62 - 1);
    if (off > 0 && off < span) { aslot_erase(K, n, k); --n; }
  }
  uint64_t offs[kMaxWormsPerInterval];
  int bad = 0;
  const int nw = sample_worms<kMaxWormsPerInterval>(st, wpts(lo, hi), p ^ q, d.SW, d.SWI, offs, &bad);
  if (bad) { d.cntA[x] = cnt_make(n, cnt_base(d.cntA[x])); return bad; }
  const uint64_t m0 = wm_above(lo);
  for (int k = 0; k < nw; ++k) {
    if (n >= d.cap) { d.cntA[x] = cnt_make(n, cnt_base(d.cntA[x])); return PMWA_ECAPACITY; }
    const uint64_t key = wkey((m0 + offs[k]) & (kTwo59 - 1), 0, p ^ 1 ^ (k & 1));
    aslot_insert(K, n, slot_lower(K, n, kpk(key)), key);
    ++n;
  }
  d.cntA[x] = cnt_make(n, n ? kab(K[n - 1]) : cnt_base(d.cntA[x]));
  return PMWA_OK;
}

__device__ __forceinline__ double fsig(int sigma, double em1) { return sigma ? -em1 : __dadd_rn(2.0, em1); }
__device__ __forceinline__ double em1_of(uint64_t I, double XW) {
  return expm1_det(__dmul_rn(-2.0, __dmul_rn(__ull2double_rn(I), XW)));
}

__global__ void k_boundary(Dev d, int dir) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int a;
  if (dir == 0) {
    if (t >= d.ndx * d.Ly) return;
    a = ((t % d.ndx) * d.dom_x + d.dom_x - 1) + d.Lx * (t / d.ndx);
  } else {
    if (t >= d.ndy * d.Lx) return;
    a = (t % d.Lx) + d.Lx * ((t / d.Lx) * d.dom_y + d.dom_y - 1);
  }
  const int b = site_step(d, a, dir, +1);
  const int tag = bond_tag(d, a, dir);
  const int bid = 2 * a + dir;
  uint64_t* KA = d.keyA + size_t(a) * d.cap;
  uint64_t* KB = d.keyA + size_t(b) * d.cap;
  Stream st;
  st.init(d.key0, d.key1, uint32_t(bid), c2_word(dir ? kBy : kBx, 0, d.replica), d.sweep);
  int rc = PMWA_OK;
  // Step 2: the bond's vertices in time order (worms move, vertices do not)
  uint64_t last = 0;
  bool any = false;
  for (;;) {
    const int nA = cnt_n(d.cntA[a]);
    int k = any ? slot_lower(KA, nA, last + 1) : 0;
    while (k < nA && ktag(KA[k]) != tag) ++k;
    if (k >= nA) break;
    const uint64_t pv = kpk(KA[k]);
    last = pv; any = true;
    Legs La, Lb;
    if (!site_legs(KA, nA, pv, &La) || !site_legs(KB, cnt_n(d.cntA[b]), pv, &Lb)) {
      rc = PMWA_EINVARIANT;
      break;
    }
    double ea_dn = 0.0, eb_dn = 0.0, ea_up, eb_up;
    if (La.single) ea_up = em1_of(kTwo59, d.XW);
    else { ea_dn = em1_of(La.Idn, d.XW); ea_up = em1_of(La.Iup, d.XW); }
    if (Lb.single) eb_up = em1_of(kTwo59, d.XW);
    else { eb_dn = em1_of(Lb.Idn, d.XW); eb_up = em1_of(Lb.Iup, d.XW); }
    double cum[16], tot = 0.0;
    int lastS = -1;
    for (int S = 0; S < 16; ++S) {
      double w = vweight(d, S);
      if (w > 0.0) {
        const int s0 = S & 1, s1 = (S >> 1) & 1, s2 = (S >> 2) & 1, s3 = (S >> 3) & 1;
        if (!La.single) w = __dmul_rn(w, fsig(La.far_dn ^ s0, ea_dn));
        if (!Lb.single) w = __dmul_rn(w, fsig(Lb.far_dn ^ s1, eb_dn));
        w = __dmul_rn(w, La.single ? fsig(s2 ^ s0, ea_up) : fsig(s2 ^ La.far_up, ea_up));
        w = __dmul_rn(w, Lb.single ? fsig(s3 ^ s1, eb_up) : fsig(s3 ^ Lb.far_up, eb_up));
        if (w > 0.0) lastS = S;
      }
      tot = __dadd_rn(tot, w);
      cum[S] = tot;
    }
    if (lastS < 0) { rc = PMWA_EINVARIANT; break; }
    const double u = __dmul_rn(__dmul_rn(__ull2double_rn(st.word() >> 11), 0x1p-53), tot);
    int Sn = lastS;
    for (int S = 0; S < 16; ++S) if (u < cum[S]) { Sn = S; break; }
    const int s0 = Sn & 1, s1 = (Sn >> 1) & 1, s2 = (Sn >> 2) & 1, s3 = (Sn >> 3) & 1;
    {
      const int ka = slot_find(KA, cnt_n(d.cntA[a]), pv), kb = slot_find(KB, cnt_n(d.cntA[b]), pv);
      if (ka < 0 || kb < 0) { rc = PMWA_EINVARIANT; break; }
      KA[ka] = (KA[ka] & ~3ull) | (uint64_t(s0) << 1) | uint64_t(s2);
      KB[kb] = (KB[kb] & ~3ull) | (uint64_t(s1) << 1) | uint64_t(s3);
    }
    if (!La.single) rc = regen_interval(d, st, a, La.plo, pv, La.far_dn, s0);
    if (!rc && !Lb.single) rc = regen_interval(d, st, b, Lb.plo, pv, Lb.far_dn, s1);
    if (!rc) rc = La.single ? regen_interval(d, st, a, pv, pv, s2, s0)
                            : regen_interval(d, st, a, pv, La.phi, s2, La.far_up);
    if (!rc) rc = Lb.single ? regen_interval(d, st, b, pv, pv, s3, s1)
                            : regen_interval(d, st, b, pv, Lb.phi, s3, Lb.far_up);
    if (rc) break;
  }
  // Step 3 on this bond: erase its diagonal vertices, lay new ones
  if (!rc) {
    int nA = cnt_n(d.cntA[a]), nB = cnt_n(d.cntA[b]);
    for (int k = nA - 1; k >= 0; --k) {
      const uint64_t key = KA[k];
      if (ktag(key) != tag || kab(key) != kbl(key)) continue;
      const int kb = slot_find(KB, nB, kpk(key));
      aslot_erase(KA, nA, k); --nA;
      if (kb < 0) { rc = PMWA_EINVARIANT; break; }
      aslot_erase(KB, nB, kb); --nB;
    }
    if (!rc && d.has_vertices) {
      Stream sv;
      sv.init(d.key0, d.key1, uint32_t(bid), c2_word(kVertex, 0, d.replica), d.sweep);
      uint64_t pos = 0;
      bool first = true;
      const int baseA = cnt_base(d.cntA[a]), baseB = cnt_base(d.cntA[b]);
      int bad = 0;
      for (;;) {
        const double E = zig_exp(sv, &bad);
        if (bad) { rc = bad; break; }
        const uint64_t g = grid_gap(E, d.SV);
        const uint64_t nxt = first ? g - 1 : pos + g;
        first = false;
        if (nxt >= kTwo59) break;
        pos = nxt;
        const uint64_t pk = (pos << 3) | uint64_t(tag);
        if (slot_find(KA, nA, pk) >= 0) continue;
        const int na = slot_state(KA, nA, baseA, pk), nb = slot_state(KB, nB, baseB, pk);
        const int si = na | (nb << 1);
        if (d.TV[si] < kTwo32) {
          const uint64_t w = sv.word();
          if ((w >> 32) >= d.TV[si]) continue;
        }
        if (nA >= d.cap || nB >= d.cap) { rc = PMWA_ECAPACITY; break; }
        aslot_insert(KA, nA, slot_lower(KA, nA, pk), (pk << 2) | (uint64_t(na) << 1) | uint64_t(na));
        ++nA;
        aslot_insert(KB, nB, slot_lower(KB, nB, pk), (pk << 2) | (uint64_t(nb) << 1) | uint64_t(nb));
        ++nB;
      }
    }
    d.cntA[a] = cnt_make(nA, nA ? kab(KA[nA - 1]) : cnt_base(d.cntA[a]));
    d.cntA[b] = cnt_make(nB, nB ? kab(KB[nB - 1]) : cnt_base(d.cntA[b]));
  }
  if (!rc && st.pos >= (uint64_t(1) << 33)) rc = PMWA_ETIMEOUT;
  if (rc) set_err(d.err, rc, 2);
}

// ---------------------------------------------------------------------------
// Launchers.
static inline int blocks_for(long long n, int bs) { return int((n + bs - 1) / bs); }

int upload_zig(const Zig& z) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_zX, z.X, sizeof z.X))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zF, z.F, sizeof z.F))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zW, z.W, sizeof z.W))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zK, z.K, sizeof z.K))) return int(e);
  if ((e = cudaMemcpyToSymbol(c_zR, &z.R, sizeof z.R))) return int(e);
  return 0;
}

int launch_boundary(const Dev& d, int dir, void* stream) {
  const long long n = dir == 0 ? (long long)d.ndx * d.Ly : (long long)d.ndy * d.Lx;
  if ((dir == 0 && d.ndx < 2) || (dir == 1 && d.ndy < 2)) return 0;
  k_boundary<<<blocks_for(n, 64), 64, 0, cudaStream_t(stream)>>>(d, dir);
  return int(cudaGetLastError());
}

int launch_step3(const Dev& d, void* stream) {
  k_step3<<<blocks_for(2LL * d.N, 128), 128, 0, cudaStream_t(stream)>>>(d);
  return int(cudaGetLastError());
}

int launch_step34_sites(const Dev& d, int regen, void* stream) {
  k_step34<<<blocks_for(d.N, 128), 128, 0, cudaStream_t(stream)>>>(d, regen);
  return int(cudaGetLastError());
}

size_t step5_smem(const Dev& d) {
  const int nsub = sb_slots_host(d.dom_x, d.sub_block, d.ndx) * sb_slots_host(d.dom_y, d.sub_block, d.ndy);
  return 256 * sizeof(uint64_t) + size_t(2 * (nsub + 1) + 4) * sizeof(int) + 16 +
         size_t(d.wcap) * sizeof(WormRef);
}

int launch_step5(const Dev& d, void* stream) {
  if (d.n_cycle <= 0) return 0;
  const size_t sm = step5_smem(d);
  cudaError_t e = cudaFuncSetAttribute(k_step5, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  if (e) return int(e);
  const int nsub = sb_slots_host(d.dom_x, d.sub_block, d.ndx) * sb_slots_host(d.dom_y, d.sub_block, d.ndy);
  int bs = ((nsub + 31) / 32) * 32;
  if (bs < 64) bs = 64;
  if (bs > 256) bs = 256;
  k_step5<<<d.ndom, bs, sm, cudaStream_t(stream)>>>(d);
  return int(cudaGetLastError());
}

int launch_measure(const Dev& d, void* stream) {
  k_measure<<<blocks_for(d.N, 256), 256, 0, cudaStream_t(stream)>>>(d);
  return int(cudaGetLastError());
}

int launch_rho(const Dev& d, int K, double* out, void* stream) {
  k_rho<<<blocks_for(d.N, 128), 128, 0, cudaStream_t(stream)>>>(d, K, out);
  return int(cudaGetLastError());
}

}  // namespace pmwa
