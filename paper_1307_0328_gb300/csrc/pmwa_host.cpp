// pmwa_host.cpp -- host side of libpmwa.so: parameter checks, the tables of
// the deterministic arithmetic, the device arena, and the sweep driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pmwa_internal.h"

using namespace pmwa;

constexpr int kKernels = 7;  // 6 = whole sweep span

struct Timed {
  int kernel;
  cudaEvent_t start, stop;
};

struct pmwa_handle {
  pmwa_params p;
  Dev d;
  cudaStream_t stream;
  uint64_t sweep;
  int rows_cap;
  int rows_pending;
  uint64_t TH[256];
  DevErr* err;
  unsigned long long* phase;  // device phase-cycle counters
  int device;                 // CUDA device current at pmwa_create
  bool broken = false;        // a kernel reported an error: configuration undefined until pmwa_import
  bool profiling = false;
  std::vector<Timed> timed;            // events of launches not yet read
  std::vector<cudaEvent_t> event_pool;  // spare events
};

namespace {

struct Derived {
  int N, ndx, ndy, ndom, dom_x, dom_y, cap, capb, wcap, poolcap;
  int ntau;  // temporal domains (1: none)
  double legs_want, mb;  // legs wanted in a domain table; mean Step-3 candidates per bond
  double d[4], D, tkink, SV, SW, XW;
  GridScale SVs, SWs, XQ;
  uint64_t TV[4], SWI;
  uint64_t TH[256];
};

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

int validate(const pmwa_params* p) {
  if (!p) return PMWA_EINVAL;
  if (p->Lx < 2 || p->Ly < 2 || p->Lx > 65536 || p->Ly > 65536) return PMWA_EINVAL;
  if ((long long)p->Lx * p->Ly > (1LL << 30)) return PMWA_EINVAL;
  if (!(p->beta > 0.0) || !(p->eta > 0.0) || !(p->t >= 0.0)) return PMWA_EINVAL;
  if (!std::isfinite(p->beta) || !std::isfinite(p->eta) || !std::isfinite(p->t) ||
      !std::isfinite(p->V) || !std::isfinite(p->mu))
    return PMWA_EINVAL;
  const int dx = p->dom_x ? p->dom_x : p->Lx, dy = p->dom_y ? p->dom_y : p->Ly;
  if (dx < 1 || dy < 1 || p->Lx % dx || p->Ly % dy) return PMWA_EINVAL;
  if (p->Lx / dx > 1 && dx < 2) return PMWA_EINVAL;
  if (p->Ly / dy > 1 && dy < 2) return PMWA_EINVAL;
  if (p->exchange_every < 1 || p->n_cycle < 0 || p->n_cycle > 4095) return PMWA_EINVAL;
  const int B = p->sub_block;
  if (B < 0 || (B & 1)) return PMWA_EINVAL;
  if (B && B < dx && dx % B) return PMWA_EINVAL;
  if (B && B < dy && dy % B) return PMWA_EINVAL;
  if (p->replica >= 65536u || p->init < 0 || p->init > 2) return PMWA_EINVAL;
  if (p->cap_site < 0 || p->cap_site > (1 << 24) || p->rows_cap < 0) return PMWA_EINVAL;
  if (p->legs_hint < 0 || p->legs_hint > (1 << 20)) return PMWA_EINVAL;
  if (p->reserved[0]) return PMWA_EINVAL;
  if (!(p->vertex_window >= 0.0 && p->vertex_window <= 1.0)) return PMWA_EINVAL;
  if (p->dom_tau < 0 || p->dom_tau > 64) return PMWA_EINVAL;
  // the gap arithmetic needs the mean grid spacings 2^59/(beta eta) and
  // 2^59/(beta D) in [2^39, 2^99]
  const double be = p->beta * p->eta;
  if (!(be >= 0x1p-40 && be <= 0x1p20)) return PMWA_EINVAL;
  const double c_off = (p->c_off < 0.0) ? 0.5 * p->t : p->c_off;
  double E[4], Emax = -INFINITY, Emin = INFINITY;
  for (int s = 0; s < 4; ++s) {
    const int na = s & 1, nb = s >> 1;
    E[s] = p->V * (double)(na * nb) - (p->mu / 4.0) * (double)(na + nb);
    Emax = std::max(Emax, E[s]);
    Emin = std::min(Emin, E[s]);
  }
  const double D = (Emax + c_off) - Emin;
  if (D > 0.0 && !(p->beta * D >= 0x1p-40 && p->beta * D <= 0x1p20)) return PMWA_EINVAL;
  return PMWA_OK;
}

// Weight of a vertex with root states S (bit l = state at the root of leg l:
// 0 = lower site below, 1 = upper site below, 2 = lower site above,
// 3 = upper site above): 0 unless particles are conserved; d(s) when the
// states do not change (diagonal), t for a kink.
double weight_of(const Derived& g, int S) {
  const int s0 = S & 1, s1 = (S >> 1) & 1, s2 = (S >> 2) & 1, s3 = (S >> 3) & 1;
  if (s0 + s1 != s2 + s3) return 0.0;
  return (s0 == s2) ? g.d[s0 | (s1 << 1)] : g.tkink;
}

// Directed loops with minimal bounce for a family with leg weights w[4]:
// with the positive weights sorted a >= b >= c (absent ones are 0),
// a <= b + c gives the bounce-free symmetric solution
//   w_ab = (a+b-c)/2, w_ac = (a+c-b)/2, w_bc = (b+c-a)/2,
// and a > b + c the one with a bounce on the largest leg
//   w_aa = a-b-c, w_ab = b, w_ac = c.
void solve_family(const double w[4], double out[4][4]) {
  int idx[4] = {0, 1, 2, 3};
  std::stable_sort(idx, idx + 4, [&](int x, int y) { return w[x] > w[y]; });
  for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) out[i][j] = 0.0;
  const int A = idx[0], Bi = idx[1], Ci = idx[2];
  const double a = w[A], b = w[Bi], c = w[Ci];
  if (a <= b + c) {
    out[A][Bi] = out[Bi][A] = ((a + b) - c) / 2.0;
    out[A][Ci] = out[Ci][A] = ((a + c) - b) / 2.0;
    out[Bi][Ci] = out[Ci][Bi] = ((b + c) - a) / 2.0;
  } else {
    out[A][A] = (a - b) - c;
    out[A][Bi] = out[Bi][A] = b;
    out[A][Ci] = out[Ci][A] = c;
  }
}

// S = f 2^e with f in [0.5, 1): m = f 2^64 (exact, 53 bits), sh = 122 - e.
GridScale grid_scale(double S) {
  int e = 0;
  const double f = std::frexp(S, &e);
  return GridScale{(uint64_t)std::ldexp(f, 64), 122 - e};
}

void derive(const pmwa_params* p, Derived* g) {
  g->dom_x = p->dom_x ? p->dom_x : p->Lx;
  g->dom_y = p->dom_y ? p->dom_y : p->Ly;
  g->N = p->Lx * p->Ly;
  g->ndx = p->Lx / g->dom_x;
  g->ndy = p->Ly / g->dom_y;
  g->ndom = g->ndx * g->ndy;
  g->ntau = p->dom_tau > 1 ? p->dom_tau : 1;
  const double c_off = (p->c_off < 0.0) ? 0.5 * p->t : p->c_off;
  // Eq. 5 per bond: E(na, nb) = V na nb - (mu/4)(na + nb)
  double E[4], Emax = -INFINITY;
  for (int s = 0; s < 4; ++s) {
    const int na = s & 1, nb = s >> 1;
    E[s] = p->V * (double)(na * nb) - (p->mu / 4.0) * (double)(na + nb);
    Emax = std::max(Emax, E[s]);
  }
  const double C = Emax + c_off;
  g->D = 0.0;
  for (int s = 0; s < 4; ++s) { g->d[s] = C - E[s]; g->D = std::max(g->D, g->d[s]); }
  for (int s = 0; s < 4; ++s)
    g->TV[s] = (g->d[s] == g->D) ? kTwo32 : (uint64_t)std::floor(g->d[s] / g->D * 0x1p32);
  g->tkink = p->t;
  g->SV = (g->D > 0.0) ? 0x1p59 / (p->beta * g->D) : INFINITY;
  g->SW = 0x1p59 / (p->beta * p->eta);
  g->SWI = (g->SW >= 0x1p62) ? kTwo62 : (uint64_t)g->SW;
  g->SWs = grid_scale(g->SW);
  g->SVs = (g->D > 0.0) ? grid_scale(g->SV) : GridScale{0, 64};
  g->XW = (p->beta * p->eta) * 0x1p-59;
  {
    int e = 0;
    const double f = std::frexp((p->beta * p->eta) * 32.0, &e);
    g->XQ = GridScale{(uint64_t)std::ldexp(f, 64), 64 - e};
  }
  for (int S = 0; S < 16; ++S)
    for (int i = 0; i < 4; ++i) {
      uint64_t* th = g->TH + (S * 4 + i) * 4;
      for (int j = 0; j < 4; ++j) th[j] = kTwo32;
      const double wi = weight_of(*g, S);
      if (wi <= 0.0) continue;
      const int T = S ^ (1 << i);  // worm inside the vertex
      double w[4], m[4][4];
      for (int l = 0; l < 4; ++l) w[l] = weight_of(*g, T ^ (1 << l));
      solve_family(w, m);
      int last = 0;
      for (int j = 0; j < 4; ++j) if (m[i][j] > 0.0) last = j;
      double cum = 0.0;
      for (int j = 0; j < 4; ++j) {
        cum = cum + m[i][j] / wi;
        th[j] = (j >= last) ? kTwo32 : (uint64_t)std::floor(cum * 0x1p32);
      }
    }
  // capacities: expected events per site ~ 4 bonds x beta (D + t) + worms
  const double mean = 4.0 * p->beta * (g->D + p->t) + 2.0 * p->beta * p->eta;
  int cap = p->cap_site ? p->cap_site : int(mean + 8.0 * std::sqrt(mean) + 24.0);
  g->cap = (cap + 7) & ~7;
  const double mb = p->beta * g->D;
  g->mb = mb;
  g->capb = (int(mb + 8.0 * std::sqrt(mb) + 16.0) + 7) & ~7;
  // shared-memory tile of one domain: legs (<= 4 bonds x beta (D + t) per
  // site), Step-3 candidates (mean beta D per bond), worms (<= beta eta per site)
  const int nds = g->dom_x * g->dom_y;
  // legs wanted in a domain's table: the bound 4 beta (D + t) per site with
  // 10 % slack, or a measured mean per site with 8 standard deviations
  if (p->legs_hint > 0) {
    const double m = double(p->legs_hint) * nds;
    g->legs_want = m + 8.0 * std::sqrt(m) + 128.0;
  } else {
    g->legs_want = 1.1 * 4.0 * p->beta * (g->D + p->t) * nds + 256.0;
  }
  // temporal boundaries sit in the leg table as delimiters
  if (g->ntau > 1) g->legs_want += double(g->ntau) * nds;
  // Step-3 candidates of a domain: a Poisson count of mean 2 nds beta D;
  // worms of a domain: mean beta eta <Q> <= beta eta nds (|<b + b+>| <= 1 a
  // site); both tables hold the mean plus 16 standard deviations (a larger
  // count stops the sweep with PMWA_ECAPACITY)
  const double mc = 2.0 * nds * mb, mw = p->beta * p->eta * nds;
  g->poolcap = int(std::min(60000.0, mc + 16.0 * std::sqrt(mc) + 128.0));
  g->wcap = int(std::min(16000.0, mw + 16.0 * std::sqrt(mw) + 128.0));
}

struct Layout {
  size_t err, TH, phase, rows, cntA, cntB, keyA, keyB, total;
};

Layout layout(const pmwa_params* p, const Derived& g) {
  Layout L;
  size_t o = 0;
  const size_t N = size_t(g.N), cap = size_t(g.cap);
  const int rows_cap = p->rows_cap ? p->rows_cap : 4096;
  L.err = o; o = align_up(o + sizeof(DevErr));
  L.TH = o; o = align_up(o + 256 * sizeof(uint64_t));
  L.phase = o; o = align_up(o + 8 * sizeof(uint64_t));
  L.rows = o; o = align_up(o + size_t(rows_cap) * sizeof(pmwa_row));
  L.cntA = o; o = align_up(o + N * sizeof(uint32_t));
  L.cntB = o; o = align_up(o + N * sizeof(uint32_t));
  L.keyA = o; o = align_up(o + N * cap * sizeof(uint64_t));
  L.keyB = o; o = align_up(o + N * cap * sizeof(uint64_t));
  L.total = o;
  return L;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? PMWA_OK : PMWA_ECUDA; }

// read and clear the device error word (synchronises the stream)
int drain_error(pmwa_handle* h) {
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PMWA_ECUDA;
  DevErr e;
  if (cudaMemcpy(&e, h->err, sizeof e, cudaMemcpyDeviceToHost) != cudaSuccess) return PMWA_ECUDA;
  if (e.code) {
    // a kernel stopped part-way: the configuration is undefined (the
    // kernels queued after it left at once) until pmwa_import restores one
    h->broken = true;
    DevErr z{0, 0};
    cudaMemcpy(h->err, &z, sizeof z, cudaMemcpyHostToDevice);
    return e.code;
  }
  return PMWA_OK;
}

cudaEvent_t take_event(pmwa_handle* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// launch `fn` on the handle's stream, bracketed by events when profiling
template <class F>
int timed_launch(pmwa_handle* h, int kernel, F fn) {
  if (!h->profiling) return fn();
  Timed t{kernel, take_event(h), take_event(h)};
  cudaEventRecord(t.start, h->stream);
  const int e = fn();
  cudaEventRecord(t.stop, h->stream);
  h->timed.push_back(t);
  return e;
}

void swap_buffers(Dev& d) {
  std::swap(d.keyA, d.keyB);
  std::swap(d.cntA, d.cntB);
}

// Steps 3..stop of one sweep on the current configuration (A -> B, swap).
int run_tile(pmwa_handle* h, int stop, bool record) {
  Dev& d = h->d;
  d.sweep = uint32_t(h->sweep);
  cudaStream_t st = h->stream;
  const int eff = (stop == 6 && !record) ? 5 : stop;
  if (eff == 6) d.row = h->rows_pending;  // rows past the pending ones are kept zeroed
  if (timed_launch(h, 1, [&] { return launch_tile(d, eff, st); })) return PMWA_ECUDA;
  if (eff == 6) h->rows_pending++;
  swap_buffers(d);
  return PMWA_OK;
}

}  // namespace

namespace pmwa {

// Ziggurat of Marsaglia and Tsang for e^-x with 256 strips of area v: the
// rightmost edge R is bisected in [7, 8] until the strips, stacked from
// (R, e^-R) upward with F[i+1] = F[i] + v / X[i], X = -ln F, close with a top
// strip of area v.
static int lay_strips(double R, Zig* z) {
  const double v = (R + 1.0) * std::exp(-R);
  double X[257], F[257];
  X[1] = R;
  F[1] = std::exp(-R);
  for (int i = 1; i < 255; ++i) {
    F[i + 1] = F[i] + v / X[i];
    if (!(F[i + 1] < 1.0)) return -1;
    X[i + 1] = -std::log(F[i + 1]);
  }
  if (X[255] * (1.0 - F[255]) < v) return -1;
  if (z) {
    z->R = R;
    z->v = v;
    X[0] = v / F[1];
    F[0] = 0.0;
    X[256] = 0.0;
    F[256] = 1.0;
    std::memcpy(z->X, X, sizeof X);
    std::memcpy(z->F, F, sizeof F);
    for (int i = 0; i < 256; ++i) {
      z->S[i] = (i == 0) ? 0.0 : (F[i] - F[i + 1]) / (X[i] - X[i + 1]);
      z->K[i] = (uint64_t)std::floor(X[i + 1] / X[i] * 0x1p53);
      z->W[i] = X[i] * 0x1p-53;
      z->XF[i] = (uint64_t)(X[i] * 0x1p58);  // exact: 53-bit X[i] >= 2^-5
    }
    z->RF = (uint64_t)(R * 0x1p58);
  }
  return 1;
}

void build_zig(Zig* z) {
  double lo = 7.0, hi = 8.0;
  while (true) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    (lay_strips(mid, nullptr) < 0 ? lo : hi) = mid;
  }
  lay_strips(hi, z);
}

}  // namespace pmwa

// ---------------------------------------------------------------------------
extern "C" {

const char* pmwa_strerror(int s) {
  switch (s) {
    case PMWA_OK: return "ok";
    case PMWA_EINVAL: return "invalid argument";
    case PMWA_ECAPACITY: return "capacity exceeded";
    case PMWA_ETIMEOUT: return "bounded device loop reached its cap";
    case PMWA_ECUDA: return "CUDA runtime error";
    case PMWA_EINVARIANT: return "configuration invariant broken";
    case PMWA_EROWS: return "measurement row buffer full";
    default: return "unknown status";
  }
}

size_t pmwa_footprint(const pmwa_params* p) {
  if (validate(p)) return 0;
  Derived g;
  derive(p, &g);
  return layout(p, g).total;
}

int pmwa_tables(const pmwa_params* p, double* d4, double* D, uint64_t* tv4, uint64_t* th256,
                double* sv, double* sw, double* zig_x, double* zig_f, double* zig_w,
                uint64_t* zig_k) {
  if (validate(p)) return PMWA_EINVAL;
  Derived g;
  derive(p, &g);
  if (d4) std::memcpy(d4, g.d, sizeof g.d);
  if (D) *D = g.D;
  if (tv4) std::memcpy(tv4, g.TV, sizeof g.TV);
  if (th256) std::memcpy(th256, g.TH, sizeof g.TH);
  if (sv) *sv = g.SV;
  if (sw) *sw = g.SW;
  if (zig_x || zig_f || zig_w || zig_k) {
    Zig z;
    build_zig(&z);
    if (zig_x) std::memcpy(zig_x, z.X, sizeof z.X);
    if (zig_f) std::memcpy(zig_f, z.F, sizeof z.F);
    if (zig_w) std::memcpy(zig_w, z.W, sizeof z.W);
    if (zig_k) std::memcpy(zig_k, z.K, sizeof z.K);
  }
  return PMWA_OK;
}

int pmwa_slot_capacity(const pmwa_params* p, int32_t* cap) {
  if (!p || !cap || validate(p)) return PMWA_EINVAL;
  Derived g;
  derive(p, &g);
  *cap = int32_t(g.cap);
  return PMWA_OK;
}

int pmwa_create(const pmwa_params* p, void* arena, size_t bytes, void* stream, pmwa_handle** out) {
  if (!out) return PMWA_EINVAL;
  *out = nullptr;
  int rc = validate(p);
  if (rc) return rc;
  Derived g;
  derive(p, &g);
  const Layout L = layout(p, g);
  if (!arena || bytes < L.total || (reinterpret_cast<uintptr_t>(arena) & (kAlign - 1))) return PMWA_EINVAL;
  static bool zig_ready = false;
  {
    Zig z;
    build_zig(&z);
    if (upload_zig(z) || upload_zig_tile(z) || upload_zig_green(z)) return PMWA_ECUDA;
    zig_ready = true;
  }
  pmwa_handle* h = new (std::nothrow) pmwa_handle();
  if (!h) return PMWA_EINVAL;
  h->p = *p;
  h->stream = static_cast<cudaStream_t>(stream);
  h->sweep = 0;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return PMWA_ECUDA; }
  h->rows_cap = p->rows_cap ? p->rows_cap : 4096;
  h->rows_pending = 0;
  std::memcpy(h->TH, g.TH, sizeof g.TH);
  char* base = static_cast<char*>(arena);
  Dev& d = h->d;
  std::memset(&d, 0, sizeof d);
  d.Lx = p->Lx; d.Ly = p->Ly; d.N = g.N;
  d.dom_x = g.dom_x; d.dom_y = g.dom_y; d.ndx = g.ndx; d.ndy = g.ndy; d.ndom = g.ndom;
  d.sub_block = p->sub_block; d.n_cycle = p->n_cycle;
  d.cap = g.cap; d.capb = g.capb; d.wcap = g.wcap; d.poolcap = g.poolcap;
  d.key0 = uint32_t(p->seed); d.key1 = uint32_t(p->seed >> 32); d.replica = p->replica;
  d.beta = p->beta; d.eta = p->eta; d.SV = g.SV; d.SW = g.SW; d.XW = g.XW; d.SWI = g.SWI;
  d.SVs = g.SVs; d.SWs = g.SWs; d.XQ = g.XQ;
  d.has_vertices = g.D > 0.0 ? 1 : 0;
  for (int s = 0; s < 4; ++s) { d.TV[s] = g.TV[s]; d.dvw[s] = g.d[s]; d.dvwf[s] = float(g.d[s]); }
  d.tkink = g.tkink;
  d.tkinkf = float(g.tkink);
  d.XWf = float(g.XW);
  d.err = reinterpret_cast<DevErr*>(base + L.err);
  d.TH = reinterpret_cast<const uint64_t*>(base + L.TH);
  d.rows = reinterpret_cast<pmwa_row*>(base + L.rows);
  d.cntA = reinterpret_cast<uint32_t*>(base + L.cntA);
  d.cntB = reinterpret_cast<uint32_t*>(base + L.cntB);
  d.keyA = reinterpret_cast<uint64_t*>(base + L.keyA);
  d.keyB = reinterpret_cast<uint64_t*>(base + L.keyB);
  d.bufk[0] = d.keyA; d.bufk[1] = d.keyB;
  d.bufc[0] = d.cntA; d.bufc[1] = d.cntB;
  d.exchange_every = p->exchange_every;
  d.zig_cap = 64;
  d.worm_tries = 128;
  d.ntau = g.ntau;
  d.win_half = (p->vertex_window >= 0.5) ? kTwo59 : uint64_t(p->vertex_window * 0x1p59);
  d.tq = kTwo59 / uint64_t(g.ntau);
  d.tr = kTwo59 % uint64_t(g.ntau);
  h->err = d.err;
  h->phase = reinterpret_cast<unsigned long long*>(base + L.phase);
  d.phase_cycles = nullptr;
  if (!plan_tile_smem(&d, g.legs_want, g.mb)) {  // a domain too large for shared memory
    delete h;
    return PMWA_EINVAL;
  }
  // initial configuration: no events; floor(N/2) occupied sites from a
  // Fisher-Yates permutation of the stream (init_seed, unit 0, init phase)
  std::vector<uint32_t> cnt(size_t(g.N), 0u);
  if (p->init == 1) {
    std::vector<int> perm(size_t(g.N));
    for (int k = 0; k < g.N; ++k) perm[size_t(k)] = k;
    const uint32_t k0 = uint32_t(p->init_seed), k1 = uint32_t(p->init_seed >> 32);
    const uint32_t c2 = kInit | (p->replica << 16);
    uint64_t pos = 0;
    for (int k = g.N - 1; k >= 1; --k, ++pos) {
      // word `pos` of the stream: Philox block pos/2, half pos&1
      uint32_t c0 = uint32_t(pos >> 1), c1 = 0, cc2 = c2, c3 = 0, a0 = k0, a1 = k1;
      for (int r = 0; r < 10; ++r) {
        const uint64_t m0 = uint64_t(0xD2511F53u) * c0, m1 = uint64_t(0xCD9E8D57u) * cc2;
        const uint32_t n0 = uint32_t(m1 >> 32) ^ c1 ^ a0, n2 = uint32_t(m0 >> 32) ^ c3 ^ a1;
        c0 = n0; c1 = uint32_t(m1); cc2 = n2; c3 = uint32_t(m0);
        a0 += 0x9E3779B9u; a1 += 0xBB67AE85u;
      }
      const uint64_t w = (pos & 1) ? (uint64_t(cc2) | (uint64_t(c3) << 32)) : (uint64_t(c0) | (uint64_t(c1) << 32));
      const int j = int((unsigned __int128)w * uint64_t(k + 1) >> 64);
      std::swap(perm[size_t(k)], perm[size_t(j)]);
    }
    for (int k = 0; k < g.N / 2; ++k) cnt[size_t(perm[size_t(k)])] = 1u << 31;
  } else if (p->init == 2) {  // checkerboard: (x + y) even occupied
    for (int s = 0; s < g.N; ++s) cnt[size_t(s)] = (((s % p->Lx) + (s / p->Lx)) & 1) ? 0u : (1u << 31);
  }
  DevErr z{0, 0};
  if (cudaMemcpy(d.err, &z, sizeof z, cudaMemcpyHostToDevice) ||
      cudaMemcpy(const_cast<uint64_t*>(d.TH), g.TH, sizeof g.TH, cudaMemcpyHostToDevice) ||
      cudaMemcpy(d.cntA, cnt.data(), cnt.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) ||
      // clears ordered on the handle's stream (which may be a non-blocking
      // one) and finished before the first launch
      cudaMemsetAsync(d.cntB, 0, cnt.size() * sizeof(uint32_t), h->stream) ||  // counts stay <= cap at all times
      cudaMemsetAsync(h->phase, 0, 8 * sizeof(uint64_t), h->stream) ||
      cudaMemsetAsync(d.rows, 0, size_t(h->rows_cap) * sizeof(pmwa_row), h->stream) ||
      cudaStreamSynchronize(h->stream)) {
    delete h;
    return PMWA_ECUDA;
  }
  (void)zig_ready;
  *out = h;
  return PMWA_OK;
}

int pmwa_destroy(pmwa_handle* h) {
  if (!h) return PMWA_OK;
  cudaStreamSynchronize(h->stream);
  for (const Timed& t : h->timed) { cudaEventDestroy(t.start); cudaEventDestroy(t.stop); }
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  delete h;
  return PMWA_OK;
}

int pmwa_tile_plan(const pmwa_params* p, int32_t* smem, int32_t* legcap, int32_t* oldcap) {
  if (validate(p)) return PMWA_EINVAL;
  Derived g;
  derive(p, &g);
  Dev d;
  std::memset(&d, 0, sizeof d);
  d.Lx = p->Lx; d.Ly = p->Ly; d.dom_x = g.dom_x; d.dom_y = g.dom_y; d.ndx = g.ndx; d.ndy = g.ndy;
  d.sub_block = p->sub_block; d.wcap = g.wcap; d.poolcap = g.poolcap;
  d.ntau = g.ntau;
  d.win_half = (p->vertex_window >= 0.5) ? kTwo59 : uint64_t(p->vertex_window * 0x1p59);
  if (!plan_tile_smem(&d, g.legs_want, g.mb)) return PMWA_EINVAL;
  if (smem) *smem = d.sm_total;
  if (legcap) *legcap = d.legcap;
  if (oldcap) *oldcap = d.oldcap;
  return PMWA_OK;
}

int32_t pmwa_tile_smem(const pmwa_params* p) {
  int32_t smem = 0;
  return pmwa_tile_plan(p, &smem, nullptr, nullptr) ? 0 : smem;
}

int pmwa_set_n_cycle(pmwa_handle* h, int32_t n_cycle) {
  if (!h || n_cycle < 0 || n_cycle > 4095) return PMWA_EINVAL;
  h->d.n_cycle = n_cycle;
  h->p.n_cycle = n_cycle;
  return PMWA_OK;
}

int pmwa_set_loop_caps(pmwa_handle* h, int32_t zig_words, int32_t worm_tries) {
  if (!h || zig_words < 1 || zig_words > 64 || worm_tries < 1 || worm_tries > 128) return PMWA_EINVAL;
  h->d.zig_cap = zig_words;
  h->d.worm_tries = worm_tries;
  return PMWA_OK;
}

int pmwa_philox_blocks(pmwa_handle* h, int64_t n, const uint32_t* host_in, uint32_t* host_out) {
  if (!h || n < 0 || (n && (!host_in || !host_out))) return PMWA_EINVAL;
  if (n == 0) return PMWA_OK;
  const size_t scratch = size_t(h->d.N) * size_t(h->d.cap) * sizeof(uint64_t);
  if (size_t(n) > scratch / 40) return PMWA_EINVAL;
  uint32_t* din = reinterpret_cast<uint32_t*>(h->d.keyB);
  uint32_t* dout = din + size_t(n) * 6;
  if (cudaMemcpyAsync(din, host_in, size_t(n) * 6 * sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream) ||
      launch_philox(din, dout, n, h->stream) ||
      cudaMemcpyAsync(host_out, dout, size_t(n) * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream) ||
      cudaStreamSynchronize(h->stream))
    return PMWA_ECUDA;
  return PMWA_OK;
}

int pmwa_profile(pmwa_handle* h, int32_t enable) {
  if (!h) return PMWA_EINVAL;
  if (cudaStreamSynchronize(h->stream)) return PMWA_ECUDA;
  for (const Timed& t : h->timed) { h->event_pool.push_back(t.start); h->event_pool.push_back(t.stop); }
  h->timed.clear();
  h->profiling = enable != 0;
  h->d.phase_cycles = h->profiling ? h->phase : nullptr;
  if (cudaMemsetAsync(h->phase, 0, 8 * sizeof(uint64_t), h->stream) || cudaStreamSynchronize(h->stream))
    return PMWA_ECUDA;
  return PMWA_OK;
}

int pmwa_profile_phases(pmwa_handle* h, uint64_t* cycles, int32_t n) {
  if (!h || !cycles || n < 8) return PMWA_EINVAL;
  if (cudaStreamSynchronize(h->stream)) return PMWA_ECUDA;
  if (cudaMemcpy(cycles, h->phase, 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost)) return PMWA_ECUDA;
  if (cudaMemsetAsync(h->phase, 0, 8 * sizeof(uint64_t), h->stream) || cudaStreamSynchronize(h->stream))
    return PMWA_ECUDA;
  return PMWA_OK;
}

int pmwa_profile_read(pmwa_handle* h, double* ms, int64_t* launches, int32_t n) {
  if (!h || !ms || !launches || n < kKernels) return PMWA_EINVAL;
  if (cudaStreamSynchronize(h->stream)) return PMWA_ECUDA;
  for (int k = 0; k < n; ++k) { ms[k] = 0.0; launches[k] = 0; }
  for (const Timed& t : h->timed) {
    float e = 0.f;
    if (cudaEventElapsedTime(&e, t.start, t.stop)) return PMWA_ECUDA;
    ms[t.kernel] += e;
    launches[t.kernel] += 1;
    h->event_pool.push_back(t.start);
    h->event_pool.push_back(t.stop);
  }
  h->timed.clear();
  return PMWA_OK;
}

int pmwa_sweep(pmwa_handle* h, int64_t n) {
  if (!h || n < 0) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  if (h->rows_pending + n > h->rows_cap) return PMWA_EROWS;
  const bool multi = h->d.ndom > 1 || h->d.ntau > 1;
  for (int64_t k = 0; k < n; ++k) {
    Timed span{6, nullptr, nullptr};
    if (h->profiling) {
      span.start = take_event(h);
      span.stop = take_event(h);
      cudaEventRecord(span.start, h->stream);
    }
    if (multi && h->sweep % uint64_t(h->p.exchange_every) == 0) {
      h->d.sweep = uint32_t(h->sweep);
      const Dev& d = h->d;
      cudaStream_t st = h->stream;
      if (d.ntau > 1 && timed_launch(h, 2, [&] { return launch_temporal(d, st); })) return PMWA_ECUDA;
      if (d.ndx > 1 && timed_launch(h, 0, [&] { return launch_boundary(d, 0, st); })) return PMWA_ECUDA;
      if (d.ndy > 1 && timed_launch(h, 0, [&] { return launch_boundary(d, 1, st); })) return PMWA_ECUDA;
    }
    const int rc = run_tile(h, 6, true);
    if (rc) return rc;
    if (h->profiling) {
      cudaEventRecord(span.stop, h->stream);
      h->timed.push_back(span);
    }
    h->sweep++;
  }
  return drain_error(h);
}

int pmwa_temporal(pmwa_handle* h) {
  if (!h) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  h->d.sweep = uint32_t(h->sweep);
  if (h->d.ntau > 1 && launch_temporal(h->d, h->stream)) return PMWA_ECUDA;
  return drain_error(h);
}

int pmwa_boundary(pmwa_handle* h) {
  if (!h) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  h->d.sweep = uint32_t(h->sweep);
  if (launch_boundary(h->d, 0, h->stream) || launch_boundary(h->d, 1, h->stream)) return PMWA_ECUDA;
  return drain_error(h);
}

int pmwa_tile(pmwa_handle* h, int32_t stop) {
  if (!h || stop < 3 || stop > 6) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  if (stop == 6 && h->rows_pending + 1 > h->rows_cap) return PMWA_EROWS;
  const int rc = run_tile(h, stop, true);
  if (rc) return rc;
  return drain_error(h);
}

int pmwa_measure(pmwa_handle* h, pmwa_row* rows, int64_t max_rows, int64_t* n_rows) {
  if (!h || !n_rows || max_rows < 0 || (!rows && max_rows)) return PMWA_EINVAL;
  if (cudaStreamSynchronize(h->stream)) return PMWA_ECUDA;
  const int n = int(std::min<int64_t>(max_rows, h->rows_pending));
  if (n && cudaMemcpy(rows, h->d.rows, size_t(n) * sizeof(pmwa_row), cudaMemcpyDeviceToHost)) return PMWA_ECUDA;
  // the device keeps the fewest worms per domain as its complement, so that
  // zeroed rows and an atomic maximum give the minimum
  for (int r = 0; r < n; ++r) rows[r].w_dom_min = ~rows[r].w_dom_min;
  const int rest = h->rows_pending - n;
  if (rest > 0) {
    std::vector<pmwa_row> tail(static_cast<size_t>(rest));
    if (cudaMemcpy(tail.data(), h->d.rows + n, size_t(rest) * sizeof(pmwa_row), cudaMemcpyDeviceToHost) ||
        cudaMemcpy(h->d.rows, tail.data(), size_t(rest) * sizeof(pmwa_row), cudaMemcpyHostToDevice))
      return PMWA_ECUDA;
  }
  h->rows_pending = rest;
  // rows past the pending ones are kept zeroed (the sweeps add into them):
  // clear the n rows just freed, ordered on the handle's stream, and finish
  // before returning (a batch may launch on another stream)
  if (n && (cudaMemsetAsync(h->d.rows + rest, 0, size_t(n) * sizeof(pmwa_row), h->stream) ||
            cudaStreamSynchronize(h->stream)))
    return PMWA_ECUDA;
  *n_rows = n;
  return PMWA_OK;
}

int pmwa_rho_slices(pmwa_handle* h, int32_t K, double* host_out) {
  if (!h || K < 1 || !host_out) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  if (size_t(K) > size_t(h->d.cap)) return PMWA_EINVAL;  // scratch: the idle next-configuration slots
  double* dev = reinterpret_cast<double*>(h->d.keyB);
  if (launch_rho(h->d, K, dev, h->stream)) return PMWA_ECUDA;
  if (cudaStreamSynchronize(h->stream)) return PMWA_ECUDA;
  if (cudaMemcpy(host_out, dev, size_t(h->d.N) * size_t(K) * sizeof(double), cudaMemcpyDeviceToHost))
    return PMWA_ECUDA;
  return PMWA_OK;
}

int pmwa_green(pmwa_handle* h, int32_t K, int32_t rmax, double* gx, double* gy, double* plaq) {
  if (!h || K < 1 || rmax < 0 || !gx || !gy || !plaq) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  if (rmax > std::min(h->p.Lx, h->p.Ly) / 2) return PMWA_EINVAL;
  const size_t N = size_t(h->d.N);
  // scratch: the idle next-configuration slots hold rho, then the sums
  if (N * size_t(K) + size_t(2 * rmax + 1) > N * size_t(h->d.cap)) return PMWA_EINVAL;
  double* rho = reinterpret_cast<double*>(h->d.keyB);
  double* sums = rho + N * size_t(K);
  if (launch_rho(h->d, K, rho, h->stream)) return PMWA_ECUDA;
  if (cudaMemsetAsync(sums, 0, size_t(2 * rmax + 1) * sizeof(double), h->stream)) return PMWA_ECUDA;
  if (launch_green(h->p.Lx, h->p.Ly, K, rmax, rho, sums, h->stream)) return PMWA_ECUDA;
  std::vector<double> out(size_t(2 * rmax + 1));
  if (cudaStreamSynchronize(h->stream) ||
      cudaMemcpy(out.data(), sums, out.size() * sizeof(double), cudaMemcpyDeviceToHost))
    return PMWA_ECUDA;
  const double eta = h->p.eta, norm = double(N) * double(K);
  for (int r = 0; r < rmax; ++r) {
    gx[r] = out[size_t(r)] / norm / (eta * eta);
    gy[r] = out[size_t(rmax + r)] / norm / (eta * eta);
  }
  *plaq = out[size_t(2 * rmax)] / norm / (eta * eta * eta * eta);
  return PMWA_OK;
}

int pmwa_rho_slices_static(pmwa_handle* h, int32_t K, double* host_out) {
  if (!h) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PMWA_ECUDA;
  if (dev != h->device) return PMWA_EINVAL;  // the handle's device must be current
  if (cudaStreamSynchronize(h->stream)) return PMWA_ECUDA;
  return rho_slices_static(h->d, K, host_out, h->stream);
}

int pmwa_get_sweep(pmwa_handle* h, uint64_t* s) {
  if (!h || !s) return PMWA_EINVAL;
  *s = h->sweep;
  return PMWA_OK;
}

int pmwa_set_sweep(pmwa_handle* h, uint64_t s) {
  if (!h) return PMWA_EINVAL;
  h->sweep = s;
  return PMWA_OK;
}

int pmwa_export_bytes(pmwa_handle* h, size_t* bytes) {
  if (!h || !bytes) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  if (cudaStreamSynchronize(h->stream)) return PMWA_ECUDA;
  std::vector<uint32_t> cnt(size_t(h->d.N));
  if (cudaMemcpy(cnt.data(), h->d.cntA, cnt.size() * 4, cudaMemcpyDeviceToHost)) return PMWA_ECUDA;
  size_t n = 1 + cnt.size();
  for (uint32_t c : cnt) n += c & 0x7fffffffu;
  *bytes = n * sizeof(uint64_t);
  return PMWA_OK;
}

int pmwa_export(pmwa_handle* h, void* buf, size_t bytes) {
  size_t need = 0;
  int rc = pmwa_export_bytes(h, &need);
  if (rc) return rc;
  if (!buf || bytes < need) return PMWA_EINVAL;
  const size_t N = size_t(h->d.N), cap = size_t(h->d.cap);
  std::vector<uint32_t> cnt(N);
  std::vector<uint64_t> keys(N * cap);
  if (cudaMemcpy(cnt.data(), h->d.cntA, N * 4, cudaMemcpyDeviceToHost) ||
      cudaMemcpy(keys.data(), h->d.keyA, N * cap * 8, cudaMemcpyDeviceToHost))
    return PMWA_ECUDA;
  uint64_t* o = static_cast<uint64_t*>(buf);
  size_t k = 0;
  o[k++] = N;
  for (size_t s = 0; s < N; ++s) {
    const size_t n = cnt[s] & 0x7fffffffu;
    o[k++] = uint64_t(n) | (uint64_t(cnt[s] >> 31) << 63);
    std::memcpy(o + k, keys.data() + s * cap, n * 8);
    k += n;
  }
  return PMWA_OK;
}

int pmwa_import(pmwa_handle* h, const void* buf, size_t bytes) {
  if (!h || !buf) return PMWA_EINVAL;
  const uint64_t* in = static_cast<const uint64_t*>(buf);
  const size_t nw = bytes / 8, N = size_t(h->d.N), cap = size_t(h->d.cap);
  if (nw < 1 || in[0] != N) return PMWA_EINVAL;
  std::vector<uint32_t> cnt(N);
  std::vector<uint64_t> keys(N * cap, 0);
  size_t k = 1;
  for (size_t s = 0; s < N; ++s) {
    if (k >= nw) return PMWA_EINVAL;
    const uint64_t hd = in[k++];
    const size_t n = size_t(hd & 0x7fffffffu);
    if (n > cap) return PMWA_ECAPACITY;
    if (k + n > nw) return PMWA_EINVAL;
    for (size_t j = 0; j < n; ++j) {
      const uint64_t key = in[k + j];
      if (((key >> 2) & 7) == 6) return PMWA_EINVARIANT;
      if (j && (in[k + j - 1] >> 2) >= (key >> 2)) return PMWA_EINVARIANT;
      // continuity: state above each event = state below the next one
      const uint64_t nx = in[k + (j + 1) % n];
      const int above = int(key & 1);
      const int below_next = (((nx >> 2) & 7) == 7) ? int(1 - (nx & 1)) : int((nx >> 1) & 1);
      if (above != below_next) return PMWA_EINVARIANT;
    }
    if (n && int(hd >> 63) != int(in[k + n - 1] & 1)) return PMWA_EINVARIANT;
    std::memcpy(keys.data() + s * cap, in + k, n * 8);
    cnt[s] = uint32_t(n) | (uint32_t(hd >> 63) << 31);
    k += n;
  }
  if (cudaStreamSynchronize(h->stream) ||
      cudaMemcpy(h->d.cntA, cnt.data(), N * 4, cudaMemcpyHostToDevice) ||
      cudaMemcpy(h->d.keyA, keys.data(), N * cap * 8, cudaMemcpyHostToDevice))
    return PMWA_ECUDA;
  h->broken = false;
  return PMWA_OK;
}

int pmwa_rho_alpha(pmwa_handle* h, int32_t K, double* host_rho, int32_t* host_iv) {
  if (!h || K < 1 || !host_rho) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  const size_t N = size_t(h->d.N), per_site = size_t(K) * (2 * sizeof(double) + sizeof(int32_t));
  // scratch: the idle next-configuration slots, filled by chunks of sites
  const size_t room = N * size_t(h->d.cap) * sizeof(uint64_t);
  const size_t chunk = std::min(N, room / per_site);
  if (chunk == 0) return PMWA_EINVAL;
  double* rho = reinterpret_cast<double*>(h->d.keyB);
  int32_t* iv = host_iv ? reinterpret_cast<int32_t*>(rho + 2 * chunk * size_t(K)) : nullptr;
  for (size_t s0 = 0; s0 < N; s0 += chunk) {
    const size_t ns = std::min(chunk, N - s0), nk = ns * size_t(K);
    if (launch_rho_alpha(h->d, K, int(s0), int(ns), rho, iv, h->stream)) return PMWA_ECUDA;
    if (cudaStreamSynchronize(h->stream) ||
        cudaMemcpy(host_rho + 2 * s0 * size_t(K), rho, 2 * nk * sizeof(double), cudaMemcpyDeviceToHost) ||
        (iv && cudaMemcpy(host_iv + s0 * size_t(K), iv, nk * sizeof(int32_t), cudaMemcpyDeviceToHost)))
      return PMWA_ECUDA;
  }
  return PMWA_OK;
}

int pmwa_green_tau(pmwa_handle* h, int32_t K, int32_t rmax, double* host_g) {
  if (!h || K < 1 || K > kMaxGreenSlices || rmax < 0 || !host_g) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  if (rmax > std::min(h->p.Lx, h->p.Ly) / 2) return PMWA_EINVAL;
  const size_t N = size_t(h->d.N), NK = N * size_t(K);
  const size_t nsum = size_t(2) * size_t(rmax + 1) * size_t(K);
  // scratch: the idle next-configuration slots hold rho (rmax >= 1), then the sums
  const size_t need = ((rmax > 0 ? 2 * NK : 0) + nsum) * sizeof(double);
  if (need > N * size_t(h->d.cap) * sizeof(uint64_t)) return PMWA_EINVAL;
  double* rho = reinterpret_cast<double*>(h->d.keyB);
  double* sums = rho + (rmax > 0 ? 2 * NK : 0);
  if (launch_green_tau(h->d, K, rmax, rho, sums, h->stream)) return PMWA_ECUDA;
  std::vector<double> out(nsum);
  if (cudaStreamSynchronize(h->stream) ||
      cudaMemcpy(out.data(), sums, nsum * sizeof(double), cudaMemcpyDeviceToHost))
    return PMWA_ECUDA;
  const double eta = h->p.eta, norm = double(N) * double(K);
  for (int dir = 0; dir < 2; ++dir)
    for (int r = 0; r <= rmax; ++r)
      for (int dk = 0; dk < K; ++dk) {
        // r = 0 is the same for both directions (accumulated once, under dir 0)
        const double v = out[(size_t(r == 0 ? 0 : dir) * size_t(rmax + 1) + size_t(r)) * size_t(K) + size_t(dk)];
        host_g[(size_t(dir) * size_t(rmax + 1) + size_t(r)) * size_t(K) + size_t(dk)] = v / norm / (eta * eta);
      }
  return PMWA_OK;
}

int pmwa_npoint(pmwa_handle* h, int32_t K, int32_t n, int64_t m, const int32_t* sites, double* out) {
  if (!h || K < 1 || n < 1 || n > kMaxNpoint || m < 0 || (m > 0 && (!sites || !out))) return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  const size_t N = size_t(h->d.N);
  for (int64_t j = 0; j < m; ++j) {
    const int32_t* t = sites + size_t(j) * size_t(n);
    for (int c = 0; c < n; ++c) {
      if (t[c] < 0 || size_t(t[c]) >= N) return PMWA_EINVAL;
      for (int c2 = 0; c2 < c; ++c2)
        if (t[c2] == t[c]) return PMWA_EINVAL;  // one site twice: not a product of densities
    }
  }
  if (m == 0) return PMWA_OK;
  // scratch: the idle next-configuration slots hold rho (N K doubles), then a
  // chunk of tuples and their results
  const size_t room = N * size_t(h->d.cap) * sizeof(uint64_t), rho_bytes = N * size_t(K) * sizeof(double);
  const size_t per = size_t(n) * sizeof(int32_t) + sizeof(double);
  if (room < rho_bytes + per + 16) return PMWA_EINVAL;
  const size_t chunk = std::min(std::min(size_t(m), (room - rho_bytes - 16) / per), size_t(1) << 30);
  double* rho = reinterpret_cast<double*>(h->d.keyB);
  int32_t* tup = reinterpret_cast<int32_t*>(rho + N * size_t(K));
  double* res = reinterpret_cast<double*>(h->d.keyB) +
                (rho_bytes + ((chunk * size_t(n) * sizeof(int32_t) + 7) & ~size_t(7))) / sizeof(double);
  if (launch_rho(h->d, K, rho, h->stream)) return PMWA_ECUDA;
  for (size_t j0 = 0; j0 < size_t(m); j0 += chunk) {
    const size_t c = std::min(chunk, size_t(m) - j0);
    if (cudaStreamSynchronize(h->stream) ||
        cudaMemcpy(tup, sites + j0 * size_t(n), c * size_t(n) * sizeof(int32_t), cudaMemcpyHostToDevice) ||
        launch_npoint(K, n, int(c), rho, tup, h->p.eta, res, h->stream) || cudaStreamSynchronize(h->stream) ||
        cudaMemcpy(out + j0, res, c * sizeof(double), cudaMemcpyDeviceToHost))
      return PMWA_ECUDA;
  }
  return PMWA_OK;
}

int pmwa_npoint_alpha(pmwa_handle* h, int32_t K, int32_t n, int64_t m, const int32_t* pts, double* out) {
  if (!h || K < 1 || K > (1 << 20) || n < 1 || n > kMaxNpoint || m < 0 || (m > 0 && (!pts || !out)))
    return PMWA_EINVAL;
  if (h->broken) return PMWA_EINVARIANT;
  const int64_t N = h->d.N;
  for (int64_t j = 0; j < m; ++j) {
    const int32_t* t = pts + size_t(j) * size_t(n) * 3;
    for (int c = 0; c < n; ++c) {
      if (t[3 * c] < 0 || t[3 * c] >= N || t[3 * c + 1] < 0 || t[3 * c + 1] >= K || (t[3 * c + 2] & ~1))
        return PMWA_EINVAL;
      for (int e = 0; e < c; ++e)  // one point twice: two operators at one time on one site
        if (t[3 * e] == t[3 * c] && t[3 * e + 1] == t[3 * c + 1]) return PMWA_EINVAL;
    }
  }
  if (m == 0) return PMWA_OK;
  // scratch: the idle next-configuration slots hold a chunk of tuples and
  // their results
  const size_t room = size_t(N) * size_t(h->d.cap) * sizeof(uint64_t);
  const size_t per = size_t(n) * 3 * sizeof(int32_t) + sizeof(double);
  if (room < per + 16) return PMWA_EINVAL;
  const size_t chunk = std::min(std::min(size_t(m), (room - 16) / per), size_t(1) << 28);
  int32_t* tup = reinterpret_cast<int32_t*>(h->d.keyB);
  double* res = reinterpret_cast<double*>(h->d.keyB) + ((chunk * size_t(n) * 3 * sizeof(int32_t) + 7) / 8);
  for (size_t j0 = 0; j0 < size_t(m); j0 += chunk) {
    const size_t c = std::min(chunk, size_t(m) - j0);
    if (cudaStreamSynchronize(h->stream) ||
        cudaMemcpy(tup, pts + j0 * size_t(n) * 3, c * size_t(n) * 3 * sizeof(int32_t), cudaMemcpyHostToDevice) ||
        launch_npoint_alpha(h->d, K, n, int(c), tup, res, h->stream) || cudaStreamSynchronize(h->stream) ||
        cudaMemcpy(out + j0, res, c * sizeof(double), cudaMemcpyDeviceToHost))
      return PMWA_ECUDA;
  }
  return PMWA_OK;
}

int pmwa_check(pmwa_handle* h, int64_t* site, int32_t* what) {
  if (!h || !site || !what) return PMWA_EINVAL;
  *site = -1;
  *what = 0;
  if (h->broken) return PMWA_EINVARIANT;
  // scratch: the first idle next-configuration slot
  unsigned long long* dev = reinterpret_cast<unsigned long long*>(h->d.keyB);
  if (launch_check(h->d, dev, h->stream)) return PMWA_ECUDA;
  unsigned long long r = 0;
  if (cudaStreamSynchronize(h->stream) || cudaMemcpy(&r, dev, sizeof r, cudaMemcpyDeviceToHost))
    return PMWA_ECUDA;
  if (r == ~0ull) return PMWA_OK;
  *site = int64_t(r >> 4);
  *what = int32_t(r & 15u);
  return PMWA_EINVARIANT;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many independent instances advanced by one launch per kernel.
struct pmwa_batch {
  int n = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream for graph capture
  std::vector<pmwa_handle*> h;
  std::vector<int> active;
  std::vector<BatchBase> hbase;
  Dev* devs = nullptr;
  BatchBase* base = nullptr;
  DevErr* errs = nullptr;
  int2* tile_work = nullptr;  // grouped by launch group (see batch_group)
  int2* bwork[2] = {nullptr, nullptr};
  int n_tile = 0, n_bwork[2] = {0, 0}, cap_max = 0;
  int2* twork = nullptr;  // Step 1: blocks of sites of instances with temporal domains
  int n_twork = 0;
  int tcls_off[kBatchGroups] = {}, tcls_n[kBatchGroups] = {};
  // per launch group: work range, CTA-size class, dynamic shared memory
  int cls_off[kBatchGroups] = {}, cls_n[kBatchGroups] = {}, cls_smem[kBatchGroups] = {}, cls_thr[kBatchGroups] = {};
  int bcls_off[2][kBatchGroups] = {}, bcls_n[2][kBatchGroups] = {};
  cudaStream_t cs[kBatchGroups] = {};  // one capture branch per launch group
  cudaEvent_t fork = nullptr, join[kBatchGroups] = {};
  cudaGraphExec_t graph = nullptr;
  int graph_sweeps = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  float last_ms = 0.f;
  bool dirty = false;  // instance parameters changed since the last upload
  bool borrowed = false;               // instances belong to the caller
  std::vector<DevErr*> own_err;        // their error words, restored at destroy
};

namespace {

struct BatchLayout {
  size_t devs, base, errs, tile, bw[2], tw, tables, total;
  std::vector<size_t> inst_off, inst_bytes;
  int n_tile, n_bw[2], n_tw;
};

int boundary_bonds(const pmwa_params* p, const Derived& g, int dir) {
  if (dir == 0) return g.ndx > 1 ? g.ndx * p->Ly : 0;
  return g.ndy > 1 ? g.ndy * p->Lx : 0;
}

bool batch_layout(const pmwa_params* p, int n, BatchLayout* L) {
  if (n < 1 || n > 65536 || !p) return false;
  L->n_tile = 0; L->n_bw[0] = L->n_bw[1] = 0; L->n_tw = 0;
  L->inst_bytes.resize(size_t(n));
  L->inst_off.resize(size_t(n));
  for (int i = 0; i < n; ++i) {
    if (validate(p + i)) return false;
    if (p[i].vertex_window > 0.0) return false;  // the batch kernels run the plain vertex phase
    Derived g;
    derive(p + i, &g);
    if (g.ntau > 1) L->n_tw += g.N;  // upper bound: one site per block
    L->n_tile += g.ndom;
    for (int dir = 0; dir < 2; ++dir)
      L->n_bw[dir] += boundary_bonds(p + i, g, dir);  // upper bound: one bond per block
    L->inst_bytes[size_t(i)] = layout(p + i, g).total;
  }
  size_t o = 0;
  L->devs = o; o = align_up(o + size_t(n) * sizeof(Dev));
  L->base = o; o = align_up(o + size_t(n) * sizeof(BatchBase));
  L->errs = o; o = align_up(o + size_t(n) * sizeof(DevErr));
  L->tile = o; o = align_up(o + size_t(std::max(1, L->n_tile)) * sizeof(int2));
  for (int dir = 0; dir < 2; ++dir) { L->bw[dir] = o; o = align_up(o + size_t(std::max(1, L->n_bw[dir])) * sizeof(int2)); }
  L->tw = o; o = align_up(o + size_t(std::max(1, L->n_tw)) * sizeof(int2));
  L->tables = o;
  for (int i = 0; i < n; ++i) { L->inst_off[size_t(i)] = o; o = align_up(o + L->inst_bytes[size_t(i)]); }
  L->total = o;
  return true;
}

// Launch group of an instance: its CTA-size class (threads per CTA) and the
// number of its CTAs that fit an SM by shared memory (1, 2, 3, 4, 6 or 8+).
// A launch reserves the largest plan of its group for every CTA, so instances
// whose plans allow different residencies go to different launches: a few
// large plans then do not cut the residency of all the others.
int batch_group(const Dev& d) {
  const int c = tile_class(d.dom_x * d.dom_y, d.sm_total);
  // (1 KB the hardware reserves a CTA, up to 1 KB of static shared memory)
  const int per_sm = int((228LL * 1024) / (static_cast<long long>(d.sm_total) + 2048));
  const int r = per_sm >= 8 ? 5 : per_sm >= 6 ? 4 : per_sm >= 4 ? 3 : per_sm >= 3 ? 2 : per_sm >= 2 ? 1 : 0;
  return c * kResidencyLevels + r;
}

// work items grouped by launch group, each group in decreasing estimated
// cost, so that the longest CTAs start first
void build_tile_work(pmwa_batch* b, std::vector<int2>* work) {
  work->clear();
  for (int g = 0; g < kBatchGroups; ++g) {
    std::vector<std::pair<double, int2>> items;
    int smem = 0;
    for (int i = 0; i < b->n; ++i) {
      const Dev& d = b->h[size_t(i)]->d;
      if (batch_group(d) != g) continue;
      smem = std::max(smem, d.sm_total);
      const double cost = double(d.dom_x * d.dom_y) * b->h[size_t(i)]->p.beta *
                          (d.dvw[0] + d.tkink + 1.0) * double(d.n_cycle + 4);
      for (int k = 0; k < d.ndom; ++k) items.push_back({cost, make_int2(i, k)});
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int2>& x, const std::pair<double, int2>& y) { return x.first > y.first; });
    b->cls_off[g] = int(work->size());
    b->cls_n[g] = int(items.size());
    b->cls_smem[g] = smem;
    b->cls_thr[g] = g / kResidencyLevels;
    for (const auto& it : items) work->push_back(it.second);
  }
}

// Boundary work of both directions: blocks of bonds per instance, grouped
// by the instance's launch group, so that each group can run as its own
// chain of launches.
int build_boundary_work(pmwa_batch* b) {
  std::vector<int2> bw;
  const int bpb = boundary_bonds_per_block(b->cap_max);
  for (int dir = 0; dir < 2; ++dir) {
    bw.clear();
    for (int g = 0; g < kBatchGroups; ++g) {
      b->bcls_off[dir][g] = int(bw.size());
      for (int i = 0; i < b->n; ++i) {
        const Dev& d = b->h[size_t(i)]->d;
        if (batch_group(d) != g) continue;
        const int nb = dir == 0 ? (d.ndx > 1 ? d.ndx * d.Ly : 0) : (d.ndy > 1 ? d.ndy * d.Lx : 0);
        for (int t0 = 0; t0 < nb; t0 += bpb) bw.push_back(make_int2(i, t0));
      }
      b->bcls_n[dir][g] = int(bw.size()) - b->bcls_off[dir][g];
    }
    b->n_bwork[dir] = int(bw.size());
    if (!bw.empty() && cudaMemcpy(b->bwork[dir], bw.data(), bw.size() * sizeof(int2), cudaMemcpyHostToDevice))
      return PMWA_ECUDA;
  }
  // Step 1 of the instances with temporal domains: blocks of sites
  const int spb = temporal_sites_per_block();
  bw.clear();
  for (int g = 0; g < kBatchGroups; ++g) {
    b->tcls_off[g] = int(bw.size());
    for (int i = 0; i < b->n; ++i) {
      const Dev& d = b->h[size_t(i)]->d;
      if (batch_group(d) != g || d.ntau < 2) continue;
      for (int s0 = 0; s0 < d.N; s0 += spb) bw.push_back(make_int2(i, s0));
    }
    b->tcls_n[g] = int(bw.size()) - b->tcls_off[g];
  }
  b->n_twork = int(bw.size());
  if (!bw.empty() && cudaMemcpy(b->twork, bw.data(), bw.size() * sizeof(int2), cudaMemcpyHostToDevice))
    return PMWA_ECUDA;
  return PMWA_OK;
}

int batch_streams(pmwa_batch* b) {
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) || cudaEventCreate(&b->ev0) ||
      cudaEventCreate(&b->ev1) || cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming))
    return PMWA_ECUDA;
  for (int g = 0; g < kBatchGroups; ++g)
    if (cudaStreamCreateWithFlags(&b->cs[g], cudaStreamNonBlocking) ||
        cudaEventCreateWithFlags(&b->join[g], cudaEventDisableTiming))
      return PMWA_ECUDA;
  return PMWA_OK;
}

void batch_free_streams(pmwa_batch* b) {
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->fork) cudaEventDestroy(b->fork);
  for (int g = 0; g < kBatchGroups; ++g) {
    if (b->cs[g]) cudaStreamDestroy(b->cs[g]);
    if (b->join[g]) cudaEventDestroy(b->join[g]);
  }
  b->cap = nullptr; b->ev0 = b->ev1 = b->fork = nullptr;
  for (int g = 0; g < kBatchGroups; ++g) { b->cs[g] = nullptr; b->join[g] = nullptr; }
}

int batch_upload(pmwa_batch* b) {
  std::vector<Dev> devs(size_t(b->n));
  for (int i = 0; i < b->n; ++i) devs[size_t(i)] = b->h[size_t(i)]->d;
  std::vector<int2> tw;
  build_tile_work(b, &tw);
  if ((int)tw.size() > b->n_tile) return PMWA_EINVAL;
  if (cudaMemcpy(b->devs, devs.data(), devs.size() * sizeof(Dev), cudaMemcpyHostToDevice) ||
      cudaMemcpy(b->tile_work, tw.data(), tw.size() * sizeof(int2), cudaMemcpyHostToDevice))
    return PMWA_ECUDA;
  // the largest reservation of each CTA-size class is its kernel's allowance
  int allow[4] = {0, 0, 0, 0};
  for (int g = 0; g < kBatchGroups; ++g)
    if (b->cls_n[g]) allow[b->cls_thr[g]] = std::max(allow[b->cls_thr[g]], b->cls_smem[g]);
  for (int c = 0; c < 4; ++c)
    if (allow[c] && prepare_tile_batch(c, allow[c])) return PMWA_ECUDA;
  return PMWA_OK;
}

void batch_drop_graph(pmwa_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_sweeps = 0;
}

// One sweep of the instances of launch group g: temporal boundaries, boundary
// x, boundary y, tile.
int batch_launch_class(pmwa_batch* b, int it, int g, cudaStream_t st) {
  if (b->tcls_n[g] &&
      launch_temporal_batch(b->devs, b->base, b->twork + b->tcls_off[g], b->tcls_n[g], it, b->cap_max, st))
    return PMWA_ECUDA;
  for (int dir = 0; dir < 2; ++dir)
    if (b->bcls_n[dir][g] && launch_boundary_batch(b->devs, b->base, b->bwork[dir] + b->bcls_off[dir][g],
                                                   b->bcls_n[dir][g], it, dir, b->cap_max, st))
      return PMWA_ECUDA;
  if (b->cls_n[g] && launch_tile_batch(b->cls_thr[g], b->devs, b->base, b->tile_work + b->cls_off[g], b->cls_n[g],
                                       b->cls_smem[g], it, 6, st))
    return PMWA_ECUDA;
  return PMWA_OK;
}

int batch_launch_sweep(pmwa_batch* b, int it, cudaStream_t st) {
  if (b->n_twork && launch_temporal_batch(b->devs, b->base, b->twork, b->n_twork, it, b->cap_max, st))
    return PMWA_ECUDA;
  for (int dir = 0; dir < 2; ++dir)
    if (b->n_bwork[dir] &&
        launch_boundary_batch(b->devs, b->base, b->bwork[dir], b->n_bwork[dir], it, dir, b->cap_max, st))
      return PMWA_ECUDA;
  for (int g = kBatchGroups - 1; g >= 0; --g)
    if (b->cls_n[g] && launch_tile_batch(b->cls_thr[g], b->devs, b->base, b->tile_work + b->cls_off[g], b->cls_n[g],
                                         b->cls_smem[g], it, 6, st))
      return PMWA_ECUDA;
  return PMWA_OK;
}

}  // namespace

extern "C" {

size_t pmwa_batch_footprint(const pmwa_params* p, int32_t n) {
  BatchLayout L;
  return batch_layout(p, n, &L) ? L.total : 0;
}

int pmwa_batch_create(const pmwa_params* p, int32_t n, void* arena, size_t bytes, void* stream, pmwa_batch** out) {
  if (!out) return PMWA_EINVAL;
  *out = nullptr;
  BatchLayout L;
  if (!batch_layout(p, n, &L)) return PMWA_EINVAL;
  if (!arena || bytes < L.total || (reinterpret_cast<uintptr_t>(arena) & (kAlign - 1))) return PMWA_EINVAL;
  pmwa_batch* b = new (std::nothrow) pmwa_batch();
  if (!b) return PMWA_EINVAL;
  b->n = n;
  b->stream = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(arena);
  b->devs = reinterpret_cast<Dev*>(base + L.devs);
  b->base = reinterpret_cast<BatchBase*>(base + L.base);
  b->errs = reinterpret_cast<DevErr*>(base + L.errs);
  b->tile_work = reinterpret_cast<int2*>(base + L.tile);
  b->bwork[0] = reinterpret_cast<int2*>(base + L.bw[0]);
  b->bwork[1] = reinterpret_cast<int2*>(base + L.bw[1]);
  b->twork = reinterpret_cast<int2*>(base + L.tw);
  b->n_tile = L.n_tile;
  b->n_bwork[0] = L.n_bw[0];
  b->n_bwork[1] = L.n_bw[1];
  b->h.assign(size_t(n), nullptr);
  b->active.assign(size_t(n), 1);
  b->hbase.resize(size_t(n));
  int rc = PMWA_OK;
  for (int i = 0; i < n && rc == PMWA_OK; ++i) {
    rc = pmwa_create(p + i, base + L.inst_off[size_t(i)], L.inst_bytes[size_t(i)], stream, &b->h[size_t(i)]);
    if (rc) break;
    pmwa_handle* hi = b->h[size_t(i)];
    hi->err = hi->d.err = b->errs + i;  // one contiguous error array for the batch
    b->cap_max = std::max(b->cap_max, hi->d.cap);
  }
  if (rc == PMWA_OK && (cudaMemsetAsync(b->errs, 0, size_t(n) * sizeof(DevErr), b->stream) ||
                        cudaStreamSynchronize(b->stream)))
    rc = PMWA_ECUDA;
  if (rc == PMWA_OK) rc = build_boundary_work(b);
  if (rc == PMWA_OK) rc = batch_upload(b);
  if (rc == PMWA_OK && (prepare_boundary(b->cap_max) || prepare_temporal(b->cap_max))) rc = PMWA_ECUDA;
  if (rc == PMWA_OK) rc = batch_streams(b);
  if (rc) {
    for (pmwa_handle* hi : b->h) if (hi) pmwa_destroy(hi);
    batch_free_streams(b);
    delete b;
    return rc;
  }
  *out = b;
  return PMWA_OK;
}

size_t pmwa_batch_tables_bytes(pmwa_handle* const* hs, int32_t n) {
  if (!hs || n < 1 || n > 65536) return 0;
  int n_tile = 0, n_bw[2] = {0, 0}, n_tw = 0;
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || hs[i]->d.win_half) return 0;  // the batch kernels run the plain vertex phase
    const Dev& d = hs[i]->d;
    if (d.ntau > 1) n_tw += d.N;
    n_tile += d.ndom;
    n_bw[0] += d.ndx > 1 ? d.ndx * d.Ly : 0;
    n_bw[1] += d.ndy > 1 ? d.ndy * d.Lx : 0;
  }
  size_t o = 0;
  o = align_up(o + size_t(n) * sizeof(Dev));
  o = align_up(o + size_t(n) * sizeof(BatchBase));
  o = align_up(o + size_t(n) * sizeof(DevErr));
  o = align_up(o + size_t(std::max(1, n_tile)) * sizeof(int2));
  for (int dir = 0; dir < 2; ++dir) o = align_up(o + size_t(std::max(1, n_bw[dir])) * sizeof(int2));
  o = align_up(o + size_t(std::max(1, n_tw)) * sizeof(int2));
  return o;
}

int pmwa_batch_from_handles(pmwa_handle* const* hs, int32_t n, void* arena, size_t bytes, void* stream,
                            pmwa_batch** out) {
  if (!out) return PMWA_EINVAL;
  *out = nullptr;
  const size_t need = pmwa_batch_tables_bytes(hs, n);
  if (!need || !arena || bytes < need || (reinterpret_cast<uintptr_t>(arena) & (kAlign - 1))) return PMWA_EINVAL;
  pmwa_batch* b = new (std::nothrow) pmwa_batch();
  if (!b) return PMWA_EINVAL;
  b->n = n;
  b->borrowed = true;
  b->stream = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(arena);
  size_t o = 0;
  b->devs = reinterpret_cast<Dev*>(base + o); o = align_up(o + size_t(n) * sizeof(Dev));
  b->base = reinterpret_cast<BatchBase*>(base + o); o = align_up(o + size_t(n) * sizeof(BatchBase));
  b->errs = reinterpret_cast<DevErr*>(base + o); o = align_up(o + size_t(n) * sizeof(DevErr));
  int n_tile = 0;
  for (int i = 0; i < n; ++i) n_tile += hs[i]->d.ndom;
  b->tile_work = reinterpret_cast<int2*>(base + o); o = align_up(o + size_t(std::max(1, n_tile)) * sizeof(int2));
  b->n_tile = n_tile;
  b->h.assign(hs, hs + n);
  b->active.assign(size_t(n), 1);
  b->hbase.resize(size_t(n));
  int rc = PMWA_OK;
  for (int i = 0; i < n; ++i) {
    b->own_err.push_back(hs[i]->d.err);
    hs[i]->err = hs[i]->d.err = b->errs + i;
    b->cap_max = std::max(b->cap_max, hs[i]->d.cap);
  }
  if (cudaMemsetAsync(b->errs, 0, size_t(n) * sizeof(DevErr), b->stream) || cudaStreamSynchronize(b->stream))
    rc = PMWA_ECUDA;
  for (int dir = 0; dir < 2; ++dir) {
    b->bwork[dir] = reinterpret_cast<int2*>(base + o);
    int nb_total = 0;
    for (int i = 0; i < n; ++i) {
      const Dev& d = hs[i]->d;
      nb_total += dir == 0 ? (d.ndx > 1 ? d.ndx * d.Ly : 0) : (d.ndy > 1 ? d.ndy * d.Lx : 0);
    }
    o = align_up(o + size_t(std::max(1, nb_total)) * sizeof(int2));
  }
  b->twork = reinterpret_cast<int2*>(base + o);
  if (rc == PMWA_OK) rc = build_boundary_work(b);
  if (rc == PMWA_OK) rc = batch_upload(b);
  if (rc == PMWA_OK && (prepare_boundary(b->cap_max) || prepare_temporal(b->cap_max))) rc = PMWA_ECUDA;
  if (rc == PMWA_OK) rc = batch_streams(b);
  if (rc) {
    for (int i = 0; i < n; ++i) hs[i]->err = hs[i]->d.err = b->own_err[size_t(i)];
    batch_free_streams(b);
    delete b;
    return rc;
  }
  *out = b;
  return PMWA_OK;
}

int pmwa_batch_instance(pmwa_batch* b, int32_t i, pmwa_handle** h) {
  if (!b || !h || i < 0 || i >= b->n) return PMWA_EINVAL;
  *h = b->h[size_t(i)];
  return PMWA_OK;
}

int pmwa_batch_set_active(pmwa_batch* b, int32_t i, int32_t on) {
  if (!b || i < 0 || i >= b->n) return PMWA_EINVAL;
  b->active[size_t(i)] = on ? 1 : 0;
  return PMWA_OK;
}

int pmwa_batch_set_n_cycle(pmwa_batch* b, int32_t i, int32_t n_cycle) {
  if (!b || i < 0 || i >= b->n || n_cycle < 0 || n_cycle > 4095) return PMWA_EINVAL;
  b->h[size_t(i)]->d.n_cycle = n_cycle;
  b->h[size_t(i)]->p.n_cycle = n_cycle;
  batch_drop_graph(b);
  b->dirty = true;  // uploaded before the next batched sweep or capture
  return PMWA_OK;
}

int pmwa_batch_graph(pmwa_batch* b, int32_t sweeps) {
  if (!b || sweeps < 0 || sweeps > 4096) return PMWA_EINVAL;
  batch_drop_graph(b);
  if (sweeps == 0) return PMWA_OK;
  if (b->dirty) {
    if (cudaStreamSynchronize(b->stream)) return PMWA_ECUDA;
    const int rc = batch_upload(b);
    if (rc) return rc;
    b->dirty = false;
  }
  // one branch per launch group: the groups hold different instances, so
  // each runs its S sweeps as its own chain of launches and their tails
  // overlap; the branches join before the advance kernel
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) return PMWA_ECUDA;
  int rc = PMWA_OK;
  if (cudaEventRecord(b->fork, b->cap)) rc = PMWA_ECUDA;
  for (int g = 0; g < kBatchGroups && rc == PMWA_OK; ++g) {
    if (!b->cls_n[g] && !b->bcls_n[0][g] && !b->bcls_n[1][g] && !b->tcls_n[g]) continue;
    if (cudaStreamWaitEvent(b->cs[g], b->fork, 0)) { rc = PMWA_ECUDA; break; }
    for (int it = 0; it < sweeps && rc == PMWA_OK; ++it) rc = batch_launch_class(b, it, g, b->cs[g]);
    if (rc == PMWA_OK && (cudaEventRecord(b->join[g], b->cs[g]) || cudaStreamWaitEvent(b->cap, b->join[g], 0)))
      rc = PMWA_ECUDA;
  }
  if (rc == PMWA_OK && launch_advance(b->base, b->n, sweeps, b->cap)) rc = PMWA_ECUDA;
  if (cudaStreamEndCapture(b->cap, &g) || rc) {
    if (g) cudaGraphDestroy(g);
    return rc ? rc : PMWA_ECUDA;
  }
  const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e) { b->graph = nullptr; return PMWA_ECUDA; }
  b->graph_sweeps = sweeps;
  return PMWA_OK;
}

int pmwa_batch_sweep(pmwa_batch* b, int64_t n) {
  if (!b || n < 0) return PMWA_EINVAL;
  if (n == 0) return PMWA_OK;
  for (int i = 0; i < b->n; ++i)
    if (b->active[size_t(i)] && b->h[size_t(i)]->broken) return PMWA_EINVARIANT;
  for (int i = 0; i < b->n; ++i)
    if (b->active[size_t(i)] && b->h[size_t(i)]->rows_pending + n > b->h[size_t(i)]->rows_cap) return PMWA_EROWS;
  for (int i = 0; i < b->n; ++i) {
    const pmwa_handle* hi = b->h[size_t(i)];
    b->hbase[size_t(i)] = BatchBase{uint32_t(hi->sweep), hi->rows_pending,
                                    hi->d.keyA == hi->d.bufk[1] ? 1 : 0, b->active[size_t(i)]};
  }
  if (cudaStreamSynchronize(b->stream)) return PMWA_ECUDA;
  if (b->dirty) {
    const int rc = batch_upload(b);
    if (rc) return rc;
    b->dirty = false;
  }
  if (cudaMemcpy(b->base, b->hbase.data(), b->hbase.size() * sizeof(BatchBase), cudaMemcpyHostToDevice))
    return PMWA_ECUDA;
  cudaEventRecord(b->ev0, b->stream);
  // A launch that fails part-way leaves the work queued before it running:
  // the instances' host state (sweep, rows, buffer parity) can then no longer
  // be trusted, so wait for that work and mark every active instance broken
  // (pmwa_import restores it).
  auto fail = [&](int code) {
    cudaStreamSynchronize(b->stream);
    for (int i = 0; i < b->n; ++i)
      if (b->active[size_t(i)]) b->h[size_t(i)]->broken = true;
    return code;
  };
  if (b->graph && n % b->graph_sweeps == 0) {
    for (int64_t r = 0; r < n / b->graph_sweeps; ++r)
      if (cudaGraphLaunch(b->graph, b->stream)) return fail(PMWA_ECUDA);
  } else {
    for (int64_t it = 0; it < n; ++it) {
      const int rc = batch_launch_sweep(b, int(it), b->stream);
      if (rc) return fail(rc);
    }
  }
  cudaEventRecord(b->ev1, b->stream);
  for (int i = 0; i < b->n; ++i) {
    if (!b->active[size_t(i)]) continue;
    pmwa_handle* hi = b->h[size_t(i)];
    hi->sweep += uint64_t(n);
    hi->rows_pending += int(n);
    if (n & 1) swap_buffers(hi->d);
  }
  if (cudaStreamSynchronize(b->stream)) return PMWA_ECUDA;
  cudaEventElapsedTime(&b->last_ms, b->ev0, b->ev1);
  std::vector<DevErr> e(size_t(b->n));
  if (cudaMemcpy(e.data(), b->errs, e.size() * sizeof(DevErr), cudaMemcpyDeviceToHost)) return PMWA_ECUDA;
  int rc = PMWA_OK;
  for (size_t i = 0; i < e.size(); ++i)
    if (e[i].code) {
      b->h[i]->broken = true;  // undefined until pmwa_import on its handle
      if (rc == PMWA_OK) rc = e[i].code;
    }
  if (rc && (cudaMemsetAsync(b->errs, 0, e.size() * sizeof(DevErr), b->stream) || cudaStreamSynchronize(b->stream)))
    return PMWA_ECUDA;
  return rc;
}

int pmwa_batch_last_ms(pmwa_batch* b, double* ms) {
  if (!b || !ms) return PMWA_EINVAL;
  *ms = b->last_ms;
  return PMWA_OK;
}

int pmwa_batch_destroy(pmwa_batch* b) {
  if (!b) return PMWA_OK;
  cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  if (b->borrowed) {
    for (size_t i = 0; i < b->h.size(); ++i) b->h[i]->err = b->h[i]->d.err = b->own_err[i];
  } else {
    for (pmwa_handle* hi : b->h) pmwa_destroy(hi);
  }
  batch_free_streams(b);
  delete b;
  return PMWA_OK;
}

}  // extern "C"
